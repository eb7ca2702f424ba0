// C ABI entry points: context lifecycle, problem upload, solve dispatch.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <new>

#include "nop_internal.cuh"

int nop_ctx::pinned(const char* name, size_t bytes, void** out) {
    if (bytes == 0) bytes = 16;
    for (auto& kv : pins) {
        if (kv.first == name) {
            if (kv.second.bytes >= bytes) {
                *out = kv.second.p;
                return NOP_OK;
            }
            // the old buffer may still feed queued copies
            NOP_CUDA_TRY(this, cudaStreamSynchronize(stream));
            cudaFreeHost(kv.second.p);
            kv.second.p = nullptr;
            kv.second.bytes = 0;
            NOP_CUDA_TRY(this, cudaMallocHost(&kv.second.p, bytes));
            kv.second.bytes = bytes;
            *out = kv.second.p;
            return NOP_OK;
        }
    }
    nop::DevBuf b;
    NOP_CUDA_TRY(this, cudaMallocHost(&b.p, bytes));
    b.bytes = bytes;
    pins.emplace_back(name, b);
    *out = b.p;
    return NOP_OK;
}

int nop_ctx::check_deferred() {
    if (!tc_err_pending) return NOP_OK;
    const int e = *tc_err_pending;
    tc_err_pending = nullptr;
    if (e) {
        set_error("trunk evaluation: tensor-core completion wait timed out");
        return NOP_ETIMEOUT;
    }
    return NOP_OK;
}

int nop_ctx::scratch(const char* name, size_t bytes, void** out) {
    if (bytes == 0) bytes = 16;
    for (auto& kv : bufs) {
        if (kv.first == name) {
            if (kv.second.bytes >= bytes) {
                *out = kv.second.p;
                return NOP_OK;
            }
            cudaFree(kv.second.p);
            kv.second.p = nullptr;
            kv.second.bytes = 0;
            cudaError_t e = cudaMalloc(&kv.second.p, bytes);
            if (e != cudaSuccess) {
                set_error(std::string("cudaMalloc ") + name + ": " + cudaGetErrorString(e));
                return NOP_ENOMEM;
            }
            kv.second.bytes = bytes;
            *out = kv.second.p;
            return NOP_OK;
        }
    }
    nop::DevBuf b;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc ") + name + ": " + cudaGetErrorString(e));
        return NOP_ENOMEM;
    }
    b.bytes = bytes;
    bufs.emplace_back(name, b);
    *out = b.p;
    return NOP_OK;
}

int nop_ctx::phase_begin(int phase) {
    if (!timing) return -1;
    // phases do not nest: an inner phase belongs to the enclosing one
    if (phase_depth++ > 0) return -2;
    Mark m;
    m.phase = phase;
    for (cudaEvent_t* e : {&m.a, &m.b}) {
        if (!event_pool.empty()) {
            *e = event_pool.back();
            event_pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            --phase_depth;
            return -1;
        }
    }
    cudaEventRecord(m.a, stream);
    marks.push_back(m);
    return (int)marks.size() - 1;
}

void nop_ctx::phase_end(int mark) {
    if (mark == -1) return;
    if (phase_depth > 0) --phase_depth;
    if (mark < 0 || mark >= (int)marks.size()) return;
    cudaEventRecord(marks[mark].b, stream);
}

namespace {

int upload(nop_ctx* ctx, const char* name, const void* src, size_t bytes, void** dst) {
    NOP_TRY(ctx->scratch(name, bytes, dst));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return NOP_OK;
}

bool finite_all(const double* a, long long n) {
    for (long long i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// Coefficient check on the device: flag = 1 if a sigma_t is not a positive
// finite number or any other coefficient is not finite.
__global__ void check_kernel(long long nt, const double* sigt, long long ns, const double* sigs,
                             long long nq, const double* src, long long nf, const double* nsf,
                             int* flag) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool bad = false;
    for (long long i = i0; i < nt; i += stride) bad |= !(sigt[i] > 0.0) || !isfinite(sigt[i]);
    for (long long i = i0; i < ns; i += stride) bad |= !isfinite(sigs[i]);
    for (long long i = i0; i < nq; i += stride) bad |= !isfinite(src[i]);
    for (long long i = i0; i < nf; i += stride) bad |= !isfinite(nsf[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// Estimated contraction of source iteration for each slab instance (one block
// per instance); feeds the scheduler's iteration guess when no earlier solve
// of the layout is known.  Per group: the collision-weighted scattering
// ratio c = sum sigma_s(g->g) / sum sigma_t(g) over the cells, times the
// diffusion-theory non-leakage probability 1 / (1 + D B^2 / sigma_t) of the
// slab's fundamental mode (D = 1 / (3 sigma_t), B = pi / (L + 2 * 0.7104 /
// sigma_t), sigma_t the instance's mean); the instance keeps the largest.
// (On the 4096-slab batch this tracks the measured iteration counts within
// about 30% rms, where the largest local ratio overestimates them 14-fold.)
__global__ void rho_kernel(int G, long long C, const long long* cell_off, const int* ncell,
                           const double* width, const double* sigt, const double* sigs,
                           double* rho, double* siga_mean) {
    __shared__ double red[2][32];
    const int b = blockIdx.x;
    double best = 0.0;
    for (int g = 0; g < G; ++g) {
        double ss = 0.0, st = 0.0;
        for (long long i = threadIdx.x; i < ncell[b]; i += blockDim.x) {
            const long long c = cell_off[b] + i;
            ss += sigs[((long long)g * G + g) * C + c];
            st += sigt[(long long)g * C + c];
        }
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
            st += __shfl_xor_sync(0xffffffffu, st, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = ss;
            red[1][threadIdx.x >> 5] = st;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ss = st = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                ss += red[0][w];
                st += red[1][w];
            }
            const double stm = st / ncell[b];
            const double Bg = M_PI / (width[b] + 2.0 * 0.7104 / stm);
            const double D = 1.0 / (3.0 * stm);
            const double r = (st > 0 ? ss / st : 0.0) / (1.0 + D * Bg * Bg / stm);
            if (r > best || g == 0) siga_mean[b] = (st - ss) / ncell[b];
            best = fmax(best, r);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) rho[b] = best;
}

// Spectral radius of source iteration per slab instance in the diffusion
// approximation (the largest over groups, in-group scattering).  An error e of
// the scalar flux goes to Lambda Sigma_s e in one source iteration, Lambda the
// flux response to an isotropic source without scattering; its P1 form is
// M = -(D u')' + Sigma_t with D = 1 / (3 Sigma_t) (harmonic face values, a
// Marshak condition J = u / 2 at a vacuum face, J = 0 at a reflective one).
// With A = M - Sigma_s (the absorption operator) and mu the largest
// eigenvalue of A^{-1} Sigma_s, M v = (1 + 1/mu) Sigma_s v, so the radius is
// mu / (1 + mu).  mu comes from inverse iteration y = A^{-1} Sigma_s v with
// the Rayleigh quotient v'Sigma_s y / v'Sigma_s v.  Every quantity stays
// positive: A is a diagonally dominant M-matrix whose elimination pivots are
// carried as p_k = t_k + |u_k|, t_k = a_k + |l_k| t_{k-1} / p_{k-1} (a_k the
// row's excess over its off-diagonal sum: absorption and face leakage), and
// the iterate of the fundamental mode is positive, so FP32 loses nothing to
// cancellation.  One warp per instance and group, lane l owning a chunk of
// ceil(I / 32) cells (rounded up to odd): each recurrence (the pivots, a
// Moebius map of t_{k-1} / p_{k-1}; forward substitution; back substitution,
// affine maps) is composed per chunk, the chunk maps are scanned across the
// lanes with shuffles, and every lane then runs its chunk from its entry
// value; four inverse iterations.  The six float arrays of an instance sit in
// shared memory, or for very long instances in `work` (six floats per cell
// and group).  On the 4096-slab batch this predicts
// the iteration counts of plain source iteration to 4.6% rms (times a fitted
// 0.94), where the mean scattering ratio times a leakage factor was off by
// 26% rms.
// SMEM: one warp per block with the instance's arrays in shared memory
// (filled by coalesced loads; odd chunks, so the lanes' strided accesses hit
// 32 different banks); otherwise four warps per block on the global `work`.
template <bool SMEM>
__global__ void __launch_bounds__(SMEM ? 32 : 128) rho_si_kernel(
    int B, int G, long long C, const long long* cell_off, const int* ncell, const double* width,
    const double* sigt, const double* sigs, int refl0, int reflL, float* work, double* rho) {
    const unsigned FULL = 0xffffffffu;
    extern __shared__ float rs_sm[];
    const int lane = threadIdx.x & 31;
    const int e = SMEM ? (int)blockIdx.x : (int)blockIdx.x * 4 + (int)(threadIdx.x >> 5);
    if (e >= B * G) return;   // uniform over the warp
    const int b = e / G, g = e % G;
    const int I = ncell[b];
    const long long o = cell_off[b];
    const double h = width[b] / I;
    const double* st = sigt + (long long)g * C + o;
    const double* ss = sigs + ((long long)g * G + g) * C + o;
    float* ipv = SMEM ? rs_sm : work + 6 * ((long long)g * C + o);   // 1 / p_k
    float* alf = ipv + I;                            // |l_k| / p_k
    float* cup = alf + I;                            // |u_k| / p_k
    float* ssf = cup + I;                            // Sigma_s
    float* v = ssf + I;                              // iterate
    float* z = v + I;                                // forward-substitution values
    // (SMEM: z first holds sigma_t, read by the pivot passes only)
    if constexpr (SMEM) {
        for (int i = lane; i < I; i += 32) {
            z[i] = (float)st[i];
            ssf[i] = (float)ss[i];
        }
        __syncwarp();
    }
    auto stv = [&](int k) { return SMEM ? z[k] : (float)st[k]; };
    const int m = ((I + 31) / 32) | 1;
    const int k0 = min(I, lane * m), k1 = min(I, k0 + m);
    // face coupling between cells i and i + 1 per unit volume, D_face / h^2
    // with the harmonic D_face = 2 / (3 (sigma_t,i + sigma_t,i+1)); a vacuum
    // face leaks (2D / (h + 4D)) / h
    const float kf = (float)(2.0 / (3.0 * h * h));
    auto leak = [&](double sg) {
        const double D = 1.0 / (3.0 * sg);
        return (float)(2.0 * D / ((h + 4.0 * D) * h));
    };
    auto coef = [&](int k, float& lo, float& up, float& a, float& ssk) {
        const float stk = stv(k);
        ssk = SMEM ? ssf[k] : (float)ss[k];
        lo = k > 0 ? kf / (stv(k - 1) + stk) : 0.0f;
        up = k < I - 1 ? kf / (stk + stv(k + 1)) : 0.0f;
        a = fmaxf(stk - ssk, 0.0f);
        if (k == 0 && !refl0) a += leak(st[0]);
        if (k == I - 1 && !reflL) a += leak(st[I - 1]);
    };
    // ---- pivots: x_k = t_k / p_k = (|l| x + a) / (|l| x + a + |u|), x_{-1} = 0
    float m00 = 1.0f, m01 = 0.0f, m10 = 0.0f, m11 = 1.0f;
    auto mnorm = [&]() {
        const float mx = fmaxf(fmaxf(m00, m01), fmaxf(m10, m11));
        if (mx > 0.0f) {
            const float r = 1.0f / mx;
            m00 *= r;
            m01 *= r;
            m10 *= r;
            m11 *= r;
        }
    };
    for (int k = k0; k < k1; ++k) {
        float lo, up, a, ssk;
        coef(k, lo, up, a, ssk);
        const float n00 = lo * m00 + a * m10, n01 = lo * m01 + a * m11;
        const float n10 = lo * m00 + (a + up) * m10, n11 = lo * m01 + (a + up) * m11;
        m00 = n00;
        m01 = n01;
        m10 = n10;
        m11 = n11;
        mnorm();
    }
    for (int d = 1; d < 32; d <<= 1) {   // inclusive prefix: later chunks on the left
        const float p00 = __shfl_up_sync(FULL, m00, d), p01 = __shfl_up_sync(FULL, m01, d);
        const float p10 = __shfl_up_sync(FULL, m10, d), p11 = __shfl_up_sync(FULL, m11, d);
        if (lane >= d) {
            const float n00 = m00 * p00 + m01 * p10, n01 = m00 * p01 + m01 * p11;
            const float n10 = m10 * p00 + m11 * p10, n11 = m10 * p01 + m11 * p11;
            m00 = n00;
            m01 = n01;
            m10 = n10;
            m11 = n11;
            mnorm();
        }
    }
    {
        const float q01 = __shfl_up_sync(FULL, m01, 1), q11 = __shfl_up_sync(FULL, m11, 1);
        float x = (lane > 0 && q11 > 0.0f) ? q01 / q11 : 0.0f;
        for (int k = k0; k < k1; ++k) {
            float lo, up, a, ssk;
            coef(k, lo, up, a, ssk);
            const float t = a + lo * x;
            const float p = t + up;
            const float ip = p > 0.0f ? 1.0f / p : 0.0f;
            ipv[k] = ip;
            alf[k] = lo * ip;
            cup[k] = up * ip;
            ssf[k] = ssk;
            v[k] = 1.0f;
            x = t * ip;
        }
    }
    // (SMEM: every lane's last read of sigma_t in z precedes the first write of z)
    __syncwarp();
    // ---- inverse iteration y = A^{-1} Sigma_s v and the Rayleigh quotient
    double mu = 0.0;
    float sc = 1.0f;
    for (int it = 0; it < 4; ++it) {
        // forward substitution z_k = alf_k z_{k-1} + Sigma_s v_k / p_k
        float A = 1.0f, Bv = 0.0f;
        for (int k = k0; k < k1; ++k) {
            const float al = alf[k];
            Bv = fmaf(al, Bv, ssf[k] * (v[k] * sc) * ipv[k]);
            A *= al;
        }
        for (int d = 1; d < 32; d <<= 1) {
            const float pA = __shfl_up_sync(FULL, A, d), pB = __shfl_up_sync(FULL, Bv, d);
            if (lane >= d) {
                Bv = fmaf(A, pB, Bv);
                A *= pA;
            }
        }
        float zc = __shfl_up_sync(FULL, Bv, 1);
        if (lane == 0) zc = 0.0f;
        for (int k = k0; k < k1; ++k) {
            zc = fmaf(alf[k], zc, ssf[k] * (v[k] * sc) * ipv[k]);
            z[k] = zc;
        }
        __syncwarp();
        // back substitution y_k = z_k + cup_k y_{k+1}, from the right
        A = 1.0f;
        Bv = 0.0f;
        for (int k = k1 - 1; k >= k0; --k) {
            const float c = cup[k];
            Bv = fmaf(c, Bv, z[k]);
            A *= c;
        }
        for (int d = 1; d < 32; d <<= 1) {
            const float pA = __shfl_down_sync(FULL, A, d), pB = __shfl_down_sync(FULL, Bv, d);
            if (lane + d < 32) {
                Bv = fmaf(A, pB, Bv);
                A *= pA;
            }
        }
        float yc = __shfl_down_sync(FULL, Bv, 1);
        if (lane == 31) yc = 0.0f;
        double num = 0.0, den = 0.0;
        float mx = 0.0f;
        for (int k = k1 - 1; k >= k0; --k) {
            yc = fmaf(cup[k], yc, z[k]);
            const float vk = v[k] * sc;
            const float sv = ssf[k] * vk;
            num += (double)(sv * yc);
            den += (double)(sv * vk);
            v[k] = yc;
            mx = fmaxf(mx, yc);
        }
        for (int d = 16; d > 0; d >>= 1) {
            num += __shfl_xor_sync(FULL, num, d);
            den += __shfl_xor_sync(FULL, den, d);
            mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, d));
        }
        __syncwarp();
        if (!(den > 0.0) || !(mx > 0.0) || !isfinite(num)) {
            mu = 0.0;
            break;
        }
        mu = num / den;
        sc = 1.0f / mx;
    }
    // no scattering: nothing to iterate; a singular absorption operator (no
    // absorption, reflective faces): the slowest possible iteration
    if (lane == 0) {
        const double r = isfinite(mu) ? mu / (1.0 + mu) : 0.9999;
        rho[e] = fmin(0.9999, fmax(0.0, r));
    }
}

}  // namespace

extern "C" {

const char* nop_status_str(int s) {
    switch (s) {
        case NOP_OK: return "ok";
        case NOP_EINVAL: return "invalid argument";
        case NOP_ECUDA: return "CUDA error";
        case NOP_ENOMEM: return "out of memory";
        case NOP_ENOCONV: return "iteration cap reached";
        case NOP_EDIVERGE: return "recast iteration diverged";
        case NOP_ETIMEOUT: return "device wait limit reached";
        case NOP_ENAN: return "non-finite value";
        case NOP_ESTATE: return "call out of order";
        case NOP_EIO: return "file input/output failed";
        default: return "unknown status";
    }
}

const char* nop_last_error(nop_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int nop_create(nop_ctx** out, int device) {
    if (!out) return NOP_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return NOP_ECUDA;
    nop_ctx* c = new (std::nothrow) nop_ctx();
    if (!c) return NOP_ENOMEM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return NOP_ECUDA;
    }
    c->stream = c->own_stream;
    *out = c;
    return NOP_OK;
}

int nop_destroy(nop_ctx* ctx) {
    if (!ctx) return NOP_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& m : ctx->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (auto& kv : ctx->bufs) cudaFree(kv.second.p);
    for (auto& kv : ctx->pins) cudaFreeHost(kv.second.p);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return NOP_OK;
}

int nop_set_stream(nop_ctx* ctx, void* stream) {
    if (!ctx) return NOP_EINVAL;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return NOP_OK;
}

int nop_sched_select_teams(int n, const double* lat_warp, const double* lat_team, int warps,
                           int team_width, int mode, double margin, int* team_out,
                           double* span_out) {
    if (n < 0 || (n > 0 && !team_out) || mode < 0 || mode > 2) return NOP_EINVAL;
    std::vector<char> team;
    const int rc = nop::sn1d_select_teams(n, lat_warp, lat_team, warps, team_width, mode, margin,
                                          team, span_out);
    if (rc != NOP_OK) return rc;
    for (int b = 0; b < n; ++b) team_out[b] = team[b];
    return NOP_OK;
}

int nop_set_wait_limit(nop_ctx* ctx, long long polls) {
    if (!ctx) return NOP_EINVAL;
    ctx->wait_limit = polls < 0 ? -1 : polls;
    return NOP_OK;
}

int nop_set_timing(nop_ctx* ctx, int enable) {
    if (!ctx) return NOP_EINVAL;
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& m : ctx->marks) {
        ctx->event_pool.push_back(m.a);
        ctx->event_pool.push_back(m.b);
    }
    ctx->marks.clear();
    ctx->phase_depth = 0;
    ctx->launches = ctx->sweep_launches = 0;
    ctx->cell_angle_updates = 0;
    ctx->timing = enable != 0;
    return NOP_OK;
}

int nop_get_timing(nop_ctx* ctx, nop_timings* out) {
    if (!ctx || !out) return NOP_EINVAL;
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double ms[3] = {0, 0, 0};
    for (auto& m : ctx->marks) {
        float t = 0;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) ms[m.phase] += t;
    }
    out->sweep_ms = ms[0];
    out->operator_ms = ms[1];
    out->setup_ms = ms[2];
    out->launches = ctx->launches;
    out->sweep_launches = ctx->sweep_launches;
    out->cell_angle_updates = ctx->cell_angle_updates;
    out->last_span_ms = ctx->trace_span_ms;
    out->last_inst_max_ms = ctx->trace_max_ms;
    out->last_inst_mean_ms = ctx->trace_mean_ms;
    out->last_block_instances = ctx->trace_big;
    out->last_direct_instances = ctx->last_direct;
    out->last_tune_ms = ctx->last_tune_ms;
    return NOP_OK;
}

int nop_get_trace(nop_ctx* ctx, int n, double* start_ms, double* duration_ms, int* block_path) {
    if (!ctx || n < 0) return NOP_EINVAL;
    if ((size_t)n * 3 != ctx->trace_inst.size()) {
        ctx->set_error("no per-instance trace of that size (time a slab solve first)");
        return NOP_ESTATE;
    }
    for (int b = 0; b < n; ++b) {
        if (start_ms) start_ms[b] = ctx->trace_inst[3 * b];
        if (duration_ms) duration_ms[b] = ctx->trace_inst[3 * b + 1];
        if (block_path) block_path[b] = ctx->trace_inst[3 * b + 2] != 0.0;
    }
    return NOP_OK;
}

int nop_set_problem(nop_ctx* ctx, const nop_problem* p) {
    if (!ctx || !p) return NOP_EINVAL;
    NOP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    ctx->has_problem = false;
    ctx->diffusion = false;
    const int G = p->n_groups;
    if (G < 1 || G > 64) {
        ctx->set_error("n_groups must be in 1..64");
        return NOP_EINVAL;
    }
    if (!p->sigma_t || !p->sigma_s || !p->order) {
        ctx->set_error("sigma_t, sigma_s and order are required");
        return NOP_EINVAL;
    }
    const bool fixed = p->source != nullptr;
    const bool fiss = p->nu_sigma_f != nullptr;
    if (fiss && !p->chi) {
        ctx->set_error("chi is required with nu_sigma_f");
        return NOP_EINVAL;
    }
    long long C = 0;
    if (p->geometry == NOP_GEOM_SLAB) {
        if (p->n_inst < 1 || !p->n_cells || !p->width) {
            ctx->set_error("slab batch needs n_inst >= 1, n_cells and width");
            return NOP_EINVAL;
        }
        for (int b = 0; b < p->n_inst; ++b) {
            if (p->n_cells[b] < 1 || !(p->width[b] > 0) || p->order[b] < 2 ||
                p->order[b] > 128 || (p->order[b] & 1)) {
                ctx->set_error("slab instance " + std::to_string(b) +
                               ": need n_cells >= 1, width > 0, even order in 2..128");
                return NOP_EINVAL;
            }
            C += p->n_cells[b];
        }
    } else if (p->geometry == NOP_GEOM_XY) {
        if (p->n_inst != 1 || p->nx < 1 || p->ny < 1 || !(p->lx > 0) || !(p->ly > 0) ||
            p->order[0] != 8) {
            ctx->set_error("x-y problem needs n_inst = 1, nx, ny >= 1, lx, ly > 0, order 8");
            return NOP_EINVAL;
        }
        C = (long long)p->nx * p->ny;
    } else {
        ctx->set_error("unknown geometry");
        return NOP_EINVAL;
    }
    for (int f = 0; f < 4; ++f)
        if (p->bc[f] != NOP_BC_VACUUM && p->bc[f] != NOP_BC_REFLECTIVE) {
            ctx->set_error("boundary condition must be vacuum or reflective");
            return NOP_EINVAL;
        }
    if (p->sigma_s1 && (p->geometry != NOP_GEOM_SLAB || !fixed || fiss)) {
        ctx->set_error("sigma_s1 is supported for fixed-source slab problems only");
        return NOP_EINVAL;
    }
    if (fiss && !finite_all(p->chi, G)) {
        ctx->set_error("chi must be finite");
        return NOP_EINVAL;
    }
    ctx->geometry = p->geometry;
    ctx->G = G;
    ctx->C = C;
    ctx->has_source = fixed;
    ctx->has_fission = fiss;
    for (int f = 0; f < 4; ++f) ctx->bc[f] = p->bc[f];
    void* d;
    NOP_TRY(upload(ctx, "sigt", p->sigma_t, sizeof(double) * G * C, &d));
    ctx->sigt_d = (double*)d;
    NOP_TRY(upload(ctx, "sigs", p->sigma_s, sizeof(double) * G * G * C, &d));
    ctx->sigs_d = (double*)d;
    ctx->src_d = nullptr;
    ctx->nsf_d = nullptr;
    ctx->chi_d = nullptr;
    ctx->sigs1_d = nullptr;
    if (p->sigma_s1) {
        NOP_TRY(upload(ctx, "sigs1", p->sigma_s1, sizeof(double) * G * C, &d));
        ctx->sigs1_d = (double*)d;
    }
    if (fixed) {
        NOP_TRY(upload(ctx, "src", p->source, sizeof(double) * G * C, &d));
        ctx->src_d = (double*)d;
    }
    if (fiss) {
        NOP_TRY(upload(ctx, "nsf", p->nu_sigma_f, sizeof(double) * G * C, &d));
        ctx->nsf_d = (double*)d;
        NOP_TRY(upload(ctx, "chi", p->chi, sizeof(double) * G, &d));
        ctx->chi_d = (double*)d;
    }
    // the coefficients are checked on the device, where they now are
    NOP_TRY(ctx->scratch("chk_flag", sizeof(int), &d));
    int* flag_d = (int*)d;
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(flag_d, 0, sizeof(int), ctx->stream));
    {
        const long long n = (long long)G * G * C;
        const int grid = (int)std::max<long long>(
            1, std::min<long long>((n + 255) / 256, 8LL * ctx->sm_count));
        check_kernel<<<grid, 256, 0, ctx->stream>>>(
            (long long)G * C, ctx->sigt_d, (long long)G * G * C, ctx->sigs_d,
            fixed ? (long long)G * C : 0, ctx->src_d, fiss ? (long long)G * C : 0, ctx->nsf_d,
            flag_d);
        if (ctx->sigs1_d)
            check_kernel<<<grid, 256, 0, ctx->stream>>>(0, nullptr, (long long)G * C,
                                                        ctx->sigs1_d, 0, nullptr, 0, nullptr,
                                                        flag_d);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
    }
    int bad = 0;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(&bad, flag_d, sizeof(int), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    if (p->geometry == NOP_GEOM_SLAB) {
        nop::SlabDev& s = ctx->slab;
        const int B = p->n_inst;
        // the schedule cache survives a new problem with the same batch layout
        const bool same_layout = s.n_inst == B &&
                                 std::equal(s.ncell.begin(), s.ncell.end(), p->n_cells) &&
                                 std::equal(s.order.begin(), s.order.end(), p->order) &&
                                 (int)s.last_iters.size() == B;
        if (!same_layout) {
            s.last_iters.assign(B, 0);
            s.last_iters_dsa.assign(B, 0);
            ++s.layout_version;
        }
        ++s.version;
        s.n_inst = B;
        s.C = C;
        s.ncell.assign(p->n_cells, p->n_cells + B);
        s.order.assign(p->order, p->order + B);
        s.width.assign(p->width, p->width + B);
        s.cell_off.resize(B);
        std::vector<double> dx(B);
        std::vector<long long> boff(B);
        long long o = 0, bo = 0;
        for (int b = 0; b < B; ++b) {
            s.cell_off[b] = o;
            o += s.ncell[b];
            dx[b] = s.width[b] / s.ncell[b];
            boff[b] = bo;
            bo += (long long)G * s.order[b];
        }
        s.bnd_total = bo;
        NOP_TRY(upload(ctx, "cell_off", s.cell_off.data(), sizeof(long long) * B, &d));
        s.cell_off_d = (long long*)d;
        NOP_TRY(upload(ctx, "ncell", s.ncell.data(), sizeof(int) * B, &d));
        s.ncell_d = (int*)d;
        NOP_TRY(upload(ctx, "nang", s.order.data(), sizeof(int) * B, &d));
        s.nang_d = (int*)d;
        NOP_TRY(upload(ctx, "dx", dx.data(), sizeof(double) * B, &d));
        s.dx_d = (double*)d;
        NOP_TRY(upload(ctx, "width", s.width.data(), sizeof(double) * B, &d));
        s.width_d = (double*)d;
        NOP_TRY(upload(ctx, "boff", boff.data(), sizeof(long long) * B, &d));
        s.boff_d = (long long*)d;
        NOP_TRY(ctx->scratch("rho", sizeof(double) * 2 * B, &d));
        double* rho_d = (double*)d;
        rho_kernel<<<B, 128, 0, ctx->stream>>>(G, C, s.cell_off_d, s.ncell_d, s.width_d,
                                               ctx->sigt_d, ctx->sigs_d, rho_d, rho_d + B);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        s.rho.assign(B, 0.0);
        s.siga_mean.assign(B, 0.0);
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(s.rho.data(), rho_d, sizeof(double) * B,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(s.siga_mean.data(), rho_d + B, sizeof(double) * B,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        // instances of up to about 8000 cells keep their arrays in shared
        // memory (a block each); longer batches run on a global work array
        int max_cells = 0;
        for (int b = 0; b < B; ++b) max_cells = std::max(max_cells, p->n_cells[b]);
        const size_t rs_smem = sizeof(float) * 6 * (size_t)max_cells;
        const bool rs_in_smem = rs_smem <= 192 * 1024;
        NOP_TRY(ctx->scratch("rho_si", sizeof(double) * (size_t)B * G +
                                           (rs_in_smem ? 0 : sizeof(float) * 6 * (size_t)G * C),
                             &d));
        double* rsi_d = (double*)d;
        if (rs_in_smem) {
            NOP_CUDA_TRY(ctx, cudaFuncSetAttribute(rho_si_kernel<true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)rs_smem));
            rho_si_kernel<true><<<B * G, 32, rs_smem, ctx->stream>>>(
                B, G, C, s.cell_off_d, s.ncell_d, s.width_d, ctx->sigt_d, ctx->sigs_d, ctx->bc[0],
                ctx->bc[1], nullptr, rsi_d);
        } else {
            rho_si_kernel<false><<<(B * G + 3) / 4, 128, 0, ctx->stream>>>(
                B, G, C, s.cell_off_d, s.ncell_d, s.width_d, ctx->sigt_d, ctx->sigs_d, ctx->bc[0],
                ctx->bc[1], (float*)(rsi_d + (size_t)B * G), rsi_d);
        }
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        std::vector<double> rsi((size_t)B * G);
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(rsi.data(), rsi_d, sizeof(double) * B * G,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        NOP_TRY(nop::build_gauss_legendre(ctx));   // synchronises the stream
        s.rho_si.assign(B, 0.0);
        for (int b = 0; b < B; ++b)
            for (int g = 0; g < G; ++g) s.rho_si[b] = std::max(s.rho_si[b], rsi[(size_t)b * G + g]);
    } else {
        ctx->xy.nx = p->nx;
        ctx->xy.ny = p->ny;
        ctx->xy.lx = p->lx;
        ctx->xy.ly = p->ly;
        NOP_TRY(nop::build_level_symmetric_s8(ctx));
    }
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (bad) {
        ctx->set_error("coefficients must be finite and sigma_t > 0");
        return NOP_EINVAL;
    }
    ctx->has_problem = true;
    return NOP_OK;
}

int nop_get_quadrature(nop_ctx* ctx, int inst, double* mu, double* eta, double* w,
                       int* n_out) {
    if (!ctx || !mu || !w || !n_out) return NOP_EINVAL;
    if (!ctx->has_problem) return NOP_ESTATE;
    if (ctx->geometry == NOP_GEOM_SLAB) {
        if (inst < 0 || inst >= ctx->slab.n_inst) return NOP_EINVAL;
        const int N = ctx->slab.order[inst], q = ctx->slab.qoff_h[inst];
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(mu, ctx->slab.mu_d + q, sizeof(double) * N,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(w, ctx->slab.w_d + q, sizeof(double) * N,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        *n_out = N;
    } else {
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(mu, ctx->xy.mu_d, sizeof(double) * 40,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        if (eta)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(eta, ctx->xy.eta_d, sizeof(double) * 40,
                                              cudaMemcpyDeviceToHost, ctx->stream));
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(w, ctx->xy.w_d, sizeof(double) * 40,
                                          cudaMemcpyDeviceToHost, ctx->stream));
        *n_out = 40;
    }
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

static int check_opts(nop_ctx* ctx, const nop_solve_opts* o, bool eigen) {
    if (!o) return NOP_EINVAL;
    if (!(o->tol > 0) || o->itmax < 1 || (o->precision != NOP_PREC_F32 &&
                                          o->precision != NOP_PREC_F64)) {
        ctx->set_error("need tol > 0, itmax >= 1 and a known precision");
        return NOP_EINVAL;
    }
    if (eigen && (!(o->tol_k > 0) || !(o->tol_inner > 0) || o->itmax_inner < 1)) {
        ctx->set_error("eigen solve needs tol_k, tol_inner > 0 and itmax_inner >= 1");
        return NOP_EINVAL;
    }
    if ((o->flags & NOP_DSA) && ctx->has_problem &&
        (ctx->geometry != NOP_GEOM_SLAB || ctx->sigs1_d != nullptr)) {
        ctx->set_error("diffusion synthetic acceleration: slabs with isotropic scattering only");
        return NOP_EINVAL;
    }
    return NOP_OK;
}

int nop_solve_fixed_source(nop_ctx* ctx, const nop_solve_opts* o, const double* phi0,
                           double* phi_out, nop_stats* st) {
    if (!ctx) return NOP_EINVAL;
    if (ctx->diffusion) {
        ctx->set_error("a diffusion batch is solved by nop_diffusion_solve");
        return NOP_ESTATE;
    }
    ctx->phase_depth = 0;
    NOP_TRY(check_opts(ctx, o, false));
    if (!ctx->has_problem || !ctx->has_source) {
        ctx->set_error("fixed-source solve needs a problem with a source");
        return NOP_ESTATE;
    }
    NOP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (st) {
        st->recast_iterations = 0;
        st->recast_status = NOP_OK;
    }
    bool phi0_dev = (o->flags & NOP_PHI0_DEVICE) != 0;
    const int* recast_h = nullptr;
    if (o->warm_start == NOP_WARM_RECAST) {
        // Eq. 9a / Eq. 20: the recast prediction (Eq. 24) is the initial guess
        if (!ctx->no.loaded) {
            ctx->set_error("warm start requested but no neural operator is loaded");
            return NOP_ESTATE;
        }
        if (ctx->G != 1) {
            ctx->set_error("the recast iteration needs a single-group problem");
            return NOP_EINVAL;
        }
        void* p;
        NOP_TRY(ctx->scratch("ws_phi0", sizeof(double) * ctx->C, &p));
        // enqueued without a synchronisation: the sweeps follow on the same
        // stream, and the recast statistics and the trunk kernel's wait flag
        // are read after the solve's final synchronisation
        ctx->defer_tc_check = true;
        const int rc = nop::recast_enqueue(ctx, o->recast_tol > 0 ? o->recast_tol : 1e-4,
                                           o->recast_itmax > 0 ? o->recast_itmax : 200,
                                           (double*)p, &recast_h);
        ctx->defer_tc_check = false;
        if (rc != NOP_OK) {
            ctx->tc_err_pending = nullptr;
            return rc;
        }
        phi0 = (const double*)p;
        phi0_dev = true;
    } else if (o->warm_start != NOP_WARM_NONE) {
        ctx->set_error("unknown warm start");
        return NOP_EINVAL;
    }
    int rc;
    if (ctx->geometry == NOP_GEOM_SLAB) {
        rc = nop::sn1d_solve(ctx, o, false, phi0, phi0_dev, nullptr, phi_out,
                             (o->flags & NOP_OUT_DEVICE) != 0, nullptr, st);
    } else {
        nop_solve_opts o2 = *o;
        if (phi0_dev) o2.flags |= NOP_PHI0_DEVICE;
        rc = nop::xy_solve(ctx, &o2, false, phi0, 0.0, phi_out, (o->flags & NOP_OUT_DEVICE) != 0,
                           nullptr, st);
    }
    if (recast_h) {
        NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        const int e = ctx->check_deferred();
        if (e != NOP_OK) return e;
        nop::recast_collect(ctx, recast_h, st, false);
    }
    return rc;
}

int nop_solve_eigen(nop_ctx* ctx, const nop_solve_opts* o, const double* phi0, double k0,
                    double* phi_out, double* k_out, nop_stats* st) {
    if (!ctx) return NOP_EINVAL;
    ctx->phase_depth = 0;
    NOP_TRY(check_opts(ctx, o, true));
    if (!ctx->has_problem || !ctx->has_fission) {
        ctx->set_error("eigen solve needs a problem with nu_sigma_f and chi");
        return NOP_ESTATE;
    }
    NOP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (st) {
        st->recast_iterations = 0;
        st->recast_status = NOP_OK;
    }
    const int B = ctx->geometry == NOP_GEOM_SLAB ? ctx->slab.n_inst : 1;
    std::vector<double> k0v(B, k0 > 0 ? k0 : 1.0);
    bool phi0_dev = (o->flags & NOP_PHI0_DEVICE) != 0;
    if (o->warm_start == NOP_WARM_RECAST || o->warm_start == NOP_WARM_RECAST_CP) {
        // App. A2: the simple- (Eq. A5) or constrained-preconditioning
        // (Eq. A7-A8) result seeds the model-based power iteration (Eq. A6)
        if (!ctx->no.loaded) {
            ctx->set_error("warm start requested but no neural operator is loaded");
            return NOP_ESTATE;
        }
        void* p;
        NOP_TRY(ctx->scratch("ws_phi0", sizeof(double) * ctx->G * ctx->C, &p));
        std::vector<int> sst, sit;
        NOP_TRY(nop::sp_eigen(ctx, o->recast_tol > 0 ? o->recast_tol : 1e-4,
                              o->recast_itmax > 0 ? o->recast_itmax : 200, (double*)p, &k0v, &sst,
                              &sit, o->warm_start == NOP_WARM_RECAST_CP));
        phi0 = (const double*)p;
        phi0_dev = true;
        if (st) {
            int worst = NOP_OK, imax = 0;
            for (int b = 0; b < B; ++b) {
                const int code = sst[b] == 3 ? NOP_EDIVERGE : (sst[b] == 1 ? NOP_OK : NOP_ENOCONV);
                if (code == NOP_EDIVERGE || (code != NOP_OK && worst == NOP_OK)) worst = code;
                imax = std::max(imax, sit[b]);
            }
            st->recast_iterations = imax;
            st->recast_status = worst;
        }
    } else if (o->warm_start != NOP_WARM_NONE) {
        ctx->set_error("unknown warm start");
        return NOP_EINVAL;
    }
    if (ctx->geometry == NOP_GEOM_SLAB)
        return nop::sn1d_solve(ctx, o, true, phi0, phi0_dev, k0v.data(), phi_out,
                               (o->flags & NOP_OUT_DEVICE) != 0, k_out, st);
    nop_solve_opts o2 = *o;
    if (phi0_dev) o2.flags |= NOP_PHI0_DEVICE;
    return nop::xy_solve(ctx, &o2, true, phi0, k0v[0], phi_out, (o->flags & NOP_OUT_DEVICE) != 0,
                         k_out, st);
}

}  // extern "C"
