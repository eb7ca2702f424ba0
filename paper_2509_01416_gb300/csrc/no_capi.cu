// C ABI of the neural operator: install/read parameters, raw forward, loss
// gradient, Adam training, input map, operator application, recast iteration.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nn_kernels.cuh"

using namespace nop;

namespace {

bool is_fno(const nop_ctx* ctx) {
    return ctx->no.cfg.kind == NOP_NO_FNO1D || ctx->no.cfg.kind == NOP_NO_FNO2D;
}

// Grid of the FNO for a raw call: 1D from n_coords, 2D from the current problem.
int fno_grid(nop_ctx* ctx, int n_coords, int* n1, int* n2) {
    if (ctx->no.cfg.kind == NOP_NO_FNO1D) {
        *n1 = 1;
        *n2 = n_coords;
        return NOP_OK;
    }
    if (!ctx->has_problem || ctx->geometry != NOP_GEOM_XY) {
        ctx->set_error("FNO2D calls need a current x-y problem for the grid");
        return NOP_ESTATE;
    }
    *n1 = ctx->xy.ny;
    *n2 = ctx->xy.nx;
    return NOP_OK;
}

// Upload n samples of inputs/targets and the coordinates; returns device pointers.
int stage(nop_ctx* ctx, int n, const float* inputs, const float* coords, int n_coords,
          const float* targets, int in_w, int out_w, float** U, float** X, float** Y) {
    void* p;
    NOP_TRY(ctx->scratch("no_U", sizeof(float) * (size_t)n * in_w, &p));
    *U = (float*)p;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(*U, inputs, sizeof(float) * (size_t)n * in_w,
                                      cudaMemcpyHostToDevice, ctx->stream));
    if (X) {
        NOP_TRY(ctx->scratch("no_X", sizeof(float) * (size_t)(n_coords > 0 ? n_coords : 1), &p));
        *X = (float*)p;
        if (coords && n_coords > 0)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(*X, coords, sizeof(float) * (size_t)n_coords,
                                              cudaMemcpyHostToDevice, ctx->stream));
    }
    if (Y) {
        NOP_TRY(ctx->scratch("no_Y", sizeof(float) * (size_t)n * out_w, &p));
        *Y = (float*)p;
        if (targets)
            NOP_CUDA_TRY(ctx, cudaMemcpyAsync(*Y, targets, sizeof(float) * (size_t)n * out_w,
                                              cudaMemcpyHostToDevice, ctx->stream));
    }
    return NOP_OK;
}

// forward (keep activations) + MSE + backward into ctx->no.grad; loss (device
// double) accumulated.  U/X/Y device.
int loss_grad_dev(nop_ctx* ctx, int n, const float* U, const float* X, int n_coords,
                  const float* Y, double* loss_d) {
    void* p;
    if (!is_fno(ctx)) {
        const int P = n_coords;
        NOP_TRY(ctx->scratch("no_out", sizeof(float) * (size_t)n * P, &p));
        float* out = (float*)p;
        NOP_TRY(ctx->scratch("no_dout", sizeof(float) * (size_t)n * P, &p));
        float* dout = (float*)p;
        NOP_TRY(deeponet_forward_raw(ctx, n, U, P, X, out, true));
        NOP_TRY(mse_grad(ctx, (long long)n * P, out, Y, dout, loss_d, (double)n * P));
        return deeponet_backward(ctx, n, P, dout, U, X);
    }
    int n1, n2;
    NOP_TRY(fno_grid(ctx, n_coords, &n1, &n2));
    const long long pts = (long long)n1 * n2;
    NOP_TRY(ctx->scratch("no_out", sizeof(float) * (size_t)n * pts, &p));
    float* out = (float*)p;
    NOP_TRY(ctx->scratch("no_dout", sizeof(float) * (size_t)n * pts, &p));
    float* dout = (float*)p;
    NOP_TRY(fno_forward_raw(ctx, n, U, n1, n2, out, true));
    NOP_TRY(mse_grad(ctx, (long long)n * pts, out, Y, dout, loss_d, (double)n * pts));
    return fno_backward(ctx, n, n1, n2, dout);
}

int widths(nop_ctx* ctx, int n_coords, int* in_w, int* out_w) {
    if (!is_fno(ctx)) {
        *in_w = ctx->no.cfg.sensors;
        *out_w = n_coords;
        return NOP_OK;
    }
    int n1, n2;
    NOP_TRY(fno_grid(ctx, n_coords, &n1, &n2));
    *in_w = *out_w = n1 * n2;
    return NOP_OK;
}

__global__ void gather_rows_kernel(int nb, int w, const int* idx, const float* src, float* dst) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nb * w) return;
    const int r = (int)(e / w), c = (int)(e % w);
    dst[e] = src[(long long)idx[r] * w + c];
}

// operator files: little-endian byte encoding, independent of the host
constexpr char NO_FILE_MAGIC[9] = "NOPNET01";
constexpr size_t NO_FILE_HEAD = 68;

void put_bytes(std::vector<unsigned char>& b, const char* p, size_t n) {
    b.insert(b.end(), (const unsigned char*)p, (const unsigned char*)p + n);
}

void put_le(std::vector<unsigned char>& b, uint64_t v, int nbytes) {
    for (int k = 0; k < nbytes; ++k) b.push_back((unsigned char)((v >> (8 * k)) & 0xffu));
}

uint64_t get_le(const unsigned char* p, int nbytes) {
    uint64_t v = 0;
    for (int k = 0; k < nbytes; ++k) v |= (uint64_t)p[k] << (8 * k);
    return v;
}

}  // namespace

extern "C" {

int nop_no_param_count(const nop_no_config* cfg, long long* n) {
    if (!cfg || !n) return NOP_EINVAL;
    std::vector<long long> off, len;
    return no_layout(cfg, &off, &len, n);
}

int nop_no_set(nop_ctx* ctx, const nop_no_config* cfg, const float* params) {
    if (!ctx || !cfg || !params) return NOP_EINVAL;
    NOP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    NoState& s = ctx->no;
    s.loaded = false;
    long long n;
    if (no_layout(cfg, &s.off, &s.len, &n) != NOP_OK || !(cfg->length > 0)) {
        ctx->set_error("invalid neural-operator configuration");
        return NOP_EINVAL;
    }
    s.cfg = *cfg;
    s.n_params = n;
    void* p;
    NOP_TRY(ctx->scratch("no_params", sizeof(float) * n, &p));
    s.params = (float*)p;
    NOP_TRY(ctx->scratch("no_grad", sizeof(float) * n, &p));
    s.grad = (float*)p;
    NOP_TRY(ctx->scratch("no_adam_m", sizeof(float) * n, &p));
    s.adam_m = (float*)p;
    NOP_TRY(ctx->scratch("no_adam_v", sizeof(float) * n, &p));
    s.adam_v = (float*)p;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(s.params, params, sizeof(float) * n, cudaMemcpyHostToDevice,
                                      ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(s.adam_m, 0, sizeof(float) * n, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(s.adam_v, 0, sizeof(float) * n, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    s.adam_t = 0;
    s.loaded = true;
    return NOP_OK;
}

int nop_no_get(nop_ctx* ctx, float* params) {
    if (!ctx || !params) return NOP_EINVAL;
    if (!ctx->no.loaded) return NOP_ESTATE;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(params, ctx->no.params, sizeof(float) * ctx->no.n_params,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

int nop_no_write_file(const char* path, const nop_no_config* cfg, const float* params) {
    if (!path || !cfg || !params) return NOP_EINVAL;
    long long n;
    if (nop_no_param_count(cfg, &n) != NOP_OK) return NOP_EINVAL;
    std::vector<unsigned char> head;
    put_bytes(head, NO_FILE_MAGIC, 8);
    const int ints[7] = {cfg->kind, cfg->sensors, cfg->width, cfg->basis,
                         cfg->depth, cfg->modes, cfg->proj};
    for (int v : ints) put_le(head, (uint64_t)(uint32_t)v, 4);
    for (double v : {cfg->sigma_t_star, cfg->sigma_s_star, cfg->length}) {
        uint64_t u;
        std::memcpy(&u, &v, 8);
        put_le(head, u, 8);
    }
    put_le(head, (uint64_t)n, 8);
    std::vector<unsigned char> body;
    body.reserve((size_t)n * 4);
    for (long long k = 0; k < n; ++k) {
        uint32_t u;
        std::memcpy(&u, &params[k], 4);
        put_le(body, u, 4);
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) return NOP_EIO;
    const bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size() &&
                    std::fwrite(body.data(), 1, body.size(), f) == body.size();
    const bool closed = std::fclose(f) == 0;
    return ok && closed ? NOP_OK : NOP_EIO;
}

int nop_no_read_file(const char* path, nop_no_config* cfg, float* params, long long* n_inout) {
    if (!path || !cfg || !n_inout) return NOP_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return NOP_EIO;
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    const bool err = std::ferror(f) != 0;
    std::fclose(f);
    if (err || buf.size() < NO_FILE_HEAD || std::memcmp(buf.data(), NO_FILE_MAGIC, 8) != 0)
        return NOP_EIO;
    nop_no_config c{};
    int* ints[7] = {&c.kind, &c.sensors, &c.width, &c.basis, &c.depth, &c.modes, &c.proj};
    size_t at = 8;
    for (int* v : ints) {
        *v = (int)(uint32_t)get_le(buf.data() + at, 4);
        at += 4;
    }
    for (double* v : {&c.sigma_t_star, &c.sigma_s_star, &c.length}) {
        const uint64_t u = get_le(buf.data() + at, 8);
        std::memcpy(v, &u, 8);
        at += 8;
    }
    const long long n = (long long)get_le(buf.data() + at, 8);
    at += 8;
    long long want;
    if (nop_no_param_count(&c, &want) != NOP_OK || n != want ||
        buf.size() != NO_FILE_HEAD + (size_t)n * 4)
        return NOP_EIO;
    *cfg = c;
    if (!params) {
        *n_inout = n;
        return NOP_OK;
    }
    if (*n_inout < n) return NOP_EINVAL;
    for (long long k = 0; k < n; ++k) {
        const uint32_t u = (uint32_t)get_le(buf.data() + at + 4 * k, 4);
        std::memcpy(&params[k], &u, 4);
    }
    *n_inout = n;
    return NOP_OK;
}

int nop_no_save(nop_ctx* ctx, const char* path) {
    if (!ctx || !path) return NOP_EINVAL;
    if (!ctx->no.loaded) {
        ctx->set_error("no operator to save");
        return NOP_ESTATE;
    }
    std::vector<float> p((size_t)ctx->no.n_params);
    NOP_TRY(nop_no_get(ctx, p.data()));
    const int rc = nop_no_write_file(path, &ctx->no.cfg, p.data());
    if (rc != NOP_OK) ctx->set_error(std::string("cannot write operator file ") + path);
    return rc;
}

int nop_no_load(nop_ctx* ctx, const char* path) {
    if (!ctx || !path) return NOP_EINVAL;
    nop_no_config c;
    long long n = 0;
    int rc = nop_no_read_file(path, &c, nullptr, &n);
    std::vector<float> p;
    if (rc == NOP_OK) {
        p.resize((size_t)n);
        rc = nop_no_read_file(path, &c, p.data(), &n);
    }
    if (rc != NOP_OK) {
        ctx->set_error(std::string("cannot read operator file ") + path);
        return rc;
    }
    return nop_no_set(ctx, &c, p.data());
}

int nop_no_forward(nop_ctx* ctx, int n, const float* inputs, const float* coords, int n_coords,
                   float* out) {
    if (!ctx || !inputs || !out || n < 1) return NOP_EINVAL;
    if (!ctx->no.loaded) return NOP_ESTATE;
    if (!is_fno(ctx) && (!coords || n_coords < 1)) return NOP_EINVAL;
    int in_w, out_w;
    NOP_TRY(widths(ctx, n_coords, &in_w, &out_w));
    float *U, *X;
    NOP_TRY(stage(ctx, n, inputs, coords, n_coords, nullptr, in_w, out_w, &U, &X, nullptr));
    void* p;
    NOP_TRY(ctx->scratch("no_out", sizeof(float) * (size_t)n * out_w, &p));
    float* o = (float*)p;
    if (!is_fno(ctx)) {
        NOP_TRY(deeponet_forward_raw(ctx, n, U, n_coords, X, o, false));
    } else {
        int n1, n2;
        NOP_TRY(fno_grid(ctx, n_coords, &n1, &n2));
        NOP_TRY(fno_forward_raw(ctx, n, U, n1, n2, o, false));
    }
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(out, o, sizeof(float) * (size_t)n * out_w,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

int nop_no_loss_grad(nop_ctx* ctx, int n, const float* inputs, const float* coords, int n_coords,
                     const float* targets, double* loss, float* grad) {
    if (!ctx || !inputs || !targets || !loss || !grad || n < 1) return NOP_EINVAL;
    if (!ctx->no.loaded) return NOP_ESTATE;
    if (!is_fno(ctx) && (!coords || n_coords < 1)) return NOP_EINVAL;
    int in_w, out_w;
    NOP_TRY(widths(ctx, n_coords, &in_w, &out_w));
    float *U, *X, *Y;
    NOP_TRY(stage(ctx, n, inputs, coords, n_coords, targets, in_w, out_w, &U, &X, &Y));
    void* p;
    NOP_TRY(ctx->scratch("no_loss", sizeof(double), &p));
    double* ld = (double*)p;
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(ld, 0, sizeof(double), ctx->stream));
    NOP_TRY(loss_grad_dev(ctx, n, U, X, n_coords, Y, ld));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(loss, ld, sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(grad, ctx->no.grad, sizeof(float) * ctx->no.n_params,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

int nop_no_train(nop_ctx* ctx, const nop_train_config* tc, int n, const float* inputs,
                 const float* coords, int n_coords, const float* targets, double* loss_history) {
    if (!ctx || !tc || !inputs || !targets || n < 1 || tc->steps < 1 || tc->batch < 1 ||
        tc->batch > n)
        return NOP_EINVAL;
    if (!ctx->no.loaded) return NOP_ESTATE;
    if (!is_fno(ctx) && (!coords || n_coords < 1)) return NOP_EINVAL;
    int in_w, out_w;
    NOP_TRY(widths(ctx, n_coords, &in_w, &out_w));
    // whole data set resident on the device
    void* p;
    NOP_TRY(ctx->scratch("tr_in", sizeof(float) * (size_t)n * in_w, &p));
    float* Din = (float*)p;
    NOP_TRY(ctx->scratch("tr_tg", sizeof(float) * (size_t)n * out_w, &p));
    float* Dtg = (float*)p;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(Din, inputs, sizeof(float) * (size_t)n * in_w,
                                      cudaMemcpyHostToDevice, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(Dtg, targets, sizeof(float) * (size_t)n * out_w,
                                      cudaMemcpyHostToDevice, ctx->stream));
    float* X = nullptr;
    if (coords && n_coords > 0) {
        NOP_TRY(ctx->scratch("tr_X", sizeof(float) * (size_t)n_coords, &p));
        X = (float*)p;
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(X, coords, sizeof(float) * (size_t)n_coords,
                                          cudaMemcpyHostToDevice, ctx->stream));
    }
    const int nb = tc->batch;
    std::vector<int> order((size_t)tc->steps * nb);
    for (size_t k = 0; k < order.size(); ++k)
        order[k] = tc->order ? tc->order[k] : (int)(k % (size_t)n);
    for (int v : order)
        if (v < 0 || v >= n) {
            ctx->set_error("training order index out of range");
            return NOP_EINVAL;
        }
    NOP_TRY(ctx->scratch("tr_order", sizeof(int) * order.size(), &p));
    int* ord = (int*)p;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(ord, order.data(), sizeof(int) * order.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
    NOP_TRY(ctx->scratch("tr_bin", sizeof(float) * (size_t)nb * in_w, &p));
    float* Bin = (float*)p;
    NOP_TRY(ctx->scratch("tr_btg", sizeof(float) * (size_t)nb * out_w, &p));
    float* Btg = (float*)p;
    NOP_TRY(ctx->scratch("tr_loss", sizeof(double) * tc->steps, &p));
    double* losses = (double*)p;
    NOP_CUDA_TRY(ctx, cudaMemsetAsync(losses, 0, sizeof(double) * tc->steps, ctx->stream));
    NoState& s = ctx->no;
    for (int t = 0; t < tc->steps; ++t) {
        const int* idx = ord + (size_t)t * nb;
        gather_rows_kernel<<<(int)(((long long)nb * in_w + 255) / 256), 256, 0, ctx->stream>>>(
            nb, in_w, idx, Din, Bin);
        gather_rows_kernel<<<(int)(((long long)nb * out_w + 255) / 256), 256, 0, ctx->stream>>>(
            nb, out_w, idx, Dtg, Btg);
        NOP_CUDA_TRY(ctx, cudaGetLastError());
        ctx->count_launch(false);
        ctx->count_launch(false);
        NOP_TRY(loss_grad_dev(ctx, nb, Bin, X, n_coords, Btg, losses + t));
        s.adam_t += 1;
        NOP_TRY(adam(ctx, s.n_params, s.params, s.grad, s.adam_m, s.adam_v, s.adam_t, tc->lr,
                     tc->beta1, tc->beta2, tc->eps));
    }
    if (loss_history)
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(loss_history, losses, sizeof(double) * tc->steps,
                                          cudaMemcpyDeviceToHost, ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

int nop_no_sensors(nop_ctx* ctx, const double* field, float* out) {
    if (!ctx || !field || !out) return NOP_EINVAL;
    if (!ctx->no.loaded || ctx->no.cfg.kind != NOP_NO_DEEPONET) return NOP_ESTATE;
    if (!ctx->has_problem || ctx->geometry != NOP_GEOM_SLAB) return NOP_ESTATE;
    return deeponet_project(ctx, field, out);
}

int nop_no_predict(nop_ctx* ctx, const double* src, double* phi_out) {
    if (!ctx || !src || !phi_out) return NOP_EINVAL;
    if (!ctx->no.loaded || !ctx->has_problem) return NOP_ESTATE;
    const long long C = ctx->C;
    if (ctx->G != 1) {
        ctx->set_error("operator application needs a single-group problem");
        return NOP_EINVAL;
    }
    void* p;
    NOP_TRY(ctx->scratch("pr_src", sizeof(double) * C, &p));
    double* sd = (double*)p;
    NOP_TRY(ctx->scratch("pr_phi", sizeof(double) * C, &p));
    double* pd = (double*)p;
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(sd, src, sizeof(double) * C, cudaMemcpyHostToDevice,
                                      ctx->stream));
    if (is_fno(ctx)) NOP_TRY(fno_recast(ctx, 0, 1, pd, nullptr, nullptr, true, sd));
    else NOP_TRY(deeponet_recast(ctx, 0, 1, pd, nullptr, nullptr, true, sd));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(phi_out, pd, sizeof(double) * C, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return NOP_OK;
}

}  // extern "C"

namespace nop {
// The recast iteration (Eq. 24) enqueued on the context stream: the
// prediction goes to pd (device, G*C doubles); the per-instance status and
// iteration counts (2B ints) are copied into a pinned host buffer whose
// address comes back in *stat_h, valid once the stream is synchronised.
int recast_enqueue(nop_ctx* ctx, double tol, int itmax, double* pd, const int** stat_h) {
    const int B = ctx->geometry == NOP_GEOM_SLAB ? ctx->slab.n_inst : 1;
    if (ctx->diffusion && is_fno(ctx)) {
        ctx->set_error("the diffusion recast runs with a DeepONet operator");
        return NOP_EINVAL;
    }
    void* p;
    NOP_TRY(ctx->scratch("rc_stat", sizeof(int) * 2 * B, &p));
    int* sd = (int*)p;
    if (is_fno(ctx)) NOP_TRY(fno_recast(ctx, tol, itmax, pd, sd, sd + B, false, nullptr));
    else NOP_TRY(deeponet_recast(ctx, tol, itmax, pd, sd, sd + B, false, nullptr));
    NOP_TRY(ctx->pinned("rc_stat_h", sizeof(int) * 2 * B, &p));
    NOP_CUDA_TRY(ctx, cudaMemcpyAsync(p, sd, sizeof(int) * 2 * B, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    *stat_h = (const int*)p;
    return NOP_OK;
}

// Statistics of a recast whose status buffer h (from recast_enqueue) is
// complete: per instance NOP_OK, NOP_ENOCONV (cap reached) or NOP_EDIVERGE.
void recast_collect(nop_ctx* ctx, const int* h, nop_stats* st, bool per_instance) {
    const int B = ctx->geometry == NOP_GEOM_SLAB ? ctx->slab.n_inst : 1;
    int worst = NOP_OK, imax = 0;
    for (int b = 0; b < B; ++b) {
        const int code = h[b] == 3 ? NOP_EDIVERGE : (h[b] == 0 ? NOP_ENOCONV : NOP_OK);
        if (code == NOP_EDIVERGE || (code != NOP_OK && worst == NOP_OK)) worst = code;
        imax = std::max(imax, h[B + b]);
        if (per_instance && st && st->inst_status) st->inst_status[b] = code;
        if (per_instance && st && st->inst_iterations) st->inst_iterations[b] = h[B + b];
    }
    if (st) {
        st->recast_iterations = imax;
        st->recast_status = worst;
        if (per_instance) st->status = worst;
    }
}
}  // namespace nop

extern "C" {

int nop_recast_iterate(nop_ctx* ctx, double tol, int itmax, int flags, double* phi_out,
                       nop_stats* st) {
    if (!ctx || !phi_out || !(tol > 0) || itmax < 1) return NOP_EINVAL;
    if (!ctx->no.loaded || !ctx->has_problem || !ctx->has_source) return NOP_ESTATE;
    if (ctx->G != 1) {
        ctx->set_error("the recast iteration needs a single-group problem");
        return NOP_EINVAL;
    }
    const long long C = ctx->C;
    void* p;
    double* pd = phi_out;
    if (!(flags & NOP_OUT_DEVICE)) {
        NOP_TRY(ctx->scratch("rc_phi", sizeof(double) * C, &p));
        pd = (double*)p;
    }
    const int* h = nullptr;
    NOP_TRY(nop::recast_enqueue(ctx, tol, itmax, pd, &h));
    if (!(flags & NOP_OUT_DEVICE))
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(phi_out, pd, sizeof(double) * C, cudaMemcpyDeviceToHost,
                                          ctx->stream));
    NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    nop::recast_collect(ctx, h, st, true);
    return NOP_OK;
}

int nop_sp_eigen(nop_ctx* ctx, double tol, int itmax, int flags, double* phi_out, double* k_out,
                 nop_stats* st) {
    if (!ctx || !phi_out || !k_out || !(tol > 0) || itmax < 1) return NOP_EINVAL;
    if (!ctx->no.loaded || !ctx->has_problem || !ctx->has_fission) return NOP_ESTATE;
    NOP_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    ctx->phase_depth = 0;
    const long long GC = (long long)ctx->G * ctx->C;
    double* pd = phi_out;
    void* p;
    if (!(flags & NOP_OUT_DEVICE)) {
        NOP_TRY(ctx->scratch("sp_phi", sizeof(double) * GC, &p));
        pd = (double*)p;
    }
    std::vector<double> k;
    std::vector<int> status, iters;
    NOP_TRY(sp_eigen(ctx, tol, itmax, pd, &k, &status, &iters, (flags & NOP_SP_CONSTRAINED) != 0));
    if (!(flags & NOP_OUT_DEVICE)) {
        NOP_CUDA_TRY(ctx, cudaMemcpyAsync(phi_out, pd, sizeof(double) * GC, cudaMemcpyDeviceToHost,
                                          ctx->stream));
        NOP_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    const int B = (int)k.size();
    int worst = NOP_OK, imax = 0;
    for (int b = 0; b < B; ++b) {
        k_out[b] = k[b];
        const int code = status[b] == 3 ? NOP_EDIVERGE : (status[b] == 1 ? NOP_OK : NOP_ENOCONV);
        if (code == NOP_EDIVERGE || (code != NOP_OK && worst == NOP_OK)) worst = code;
        imax = std::max(imax, iters[b]);
        if (st && st->inst_status) st->inst_status[b] = code;
        if (st && st->inst_iterations) st->inst_iterations[b] = iters[b];
    }
    if (st) {
        st->recast_iterations = imax;
        st->recast_status = worst;
        st->status = worst;
    }
    return NOP_OK;
}

}  // extern "C"
