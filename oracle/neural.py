"""FP64 neural-operator oracle: DeepONet and FNO forward/backward, MSE, Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

DeepONet (Sec. 4.1, Eq. 11; App. A1): a branch MLP maps the source sampled
at m sensors to p coefficients, a trunk MLP maps a coordinate to p basis
values, and the output is their inner product <N_T, N_B> (no output bias,
which is what the paper's parameter count of 141,200 implies).  ReLU follows
every hidden layer; the last layer of each net is linear.

FNO (Sec. 4.2; App. A1): a pointwise lift of (S(x), coordinates) to width W,
Fourier layers v <- relu(SpectralConv(v) + Linear(v)), then a two-layer
pointwise projection W -> 128 -> 1 with ReLU between (this is the layout whose
parameter count is the paper's 549,569 for W=64, 16 modes).  SpectralConv
keeps the lowest Fourier modes, multiplies them by complex in x out weight
matrices (one per mode) and transforms back; here the truncated transforms are
written out as explicit DFT sums (1D: modes k = 0..K-1 of the real FFT; 2D:
k_y in {0..m1-1} U {n_y-m1..n_y-1}, k_x in {0..m2-1}, two weight blocks).

Training (App. A1, Table A1): MSE loss and Adam.

Every function takes an optional ``quant`` hook applied to the operands of
each matrix product (identity by default).  Tests pass a bf16 rounding
function to model the CUDA kernels' operand precision; the arithmetic itself
stays FP64.
"""
import numpy as np


def _id(x):
    return x


def bf16_round(x):
    """Round an FP64 array to the nearest bfloat16 value (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------
# MLP
# ----------------------------------------------------------------------------
def mlp_forward(layers, x, quant=_id):
    """layers: list of (W[out, in], b[out]).  ReLU on all but the last layer."""
    acts = [x]
    pre = []
    h = x
    for li, (W, b) in enumerate(layers):
        z = quant(h) @ quant(W).T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(h)
    return h, (acts, pre)


def mlp_backward(layers, cache, dout, quant=_id):
    """Returns (dx, [(dW, db)]) for the MLP of mlp_forward."""
    acts, pre = cache
    grads = [None] * len(layers)
    g = dout
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        if li < len(layers) - 1:
            g = g * (pre[li] > 0)
        dW = quant(g).T @ quant(acts[li])
        db = g.sum(axis=0)
        grads[li] = (dW, db)
        g = quant(g) @ quant(W)
    return g, grads


# ----------------------------------------------------------------------------
# DeepONet
# ----------------------------------------------------------------------------
def deeponet_layers(params, net, n):
    return [(params["%s%d.W" % (net, i)], params["%s%d.b" % (net, i)]) for i in range(n)]


def deeponet_forward(params, U, X, quant=_id):
    """U: (B, m) sensor values; X: (P, d) trunk coordinates.  Returns (B, P)."""
    nb = sum(1 for k in params if k.startswith("b") and k.endswith(".W"))
    nt = sum(1 for k in params if k.startswith("t") and k.endswith(".W"))
    Bl, Tl = deeponet_layers(params, "b", nb), deeponet_layers(params, "t", nt)
    bn, cb = mlp_forward(Bl, U, quant)
    tn, ct = mlp_forward(Tl, X, quant)
    out = quant(bn) @ quant(tn).T
    return out, (bn, tn, cb, ct, nb, nt)


def deeponet_backward(params, cache, dout, quant=_id):
    bn, tn, cb, ct, nb, nt = cache
    Bl, Tl = deeponet_layers(params, "b", nb), deeponet_layers(params, "t", nt)
    dbn = quant(dout) @ quant(tn)
    dtn = quant(dout).T @ quant(bn)
    _, gb = mlp_backward(Bl, cb, dbn, quant)
    _, gt = mlp_backward(Tl, ct, dtn, quant)
    grads = {}
    for i, (dW, db) in enumerate(gb):
        grads["b%d.W" % i], grads["b%d.b" % i] = dW, db
    for i, (dW, db) in enumerate(gt):
        grads["t%d.W" % i], grads["t%d.b" % i] = dW, db
    return grads


# ----------------------------------------------------------------------------
# FNO 1D
# ----------------------------------------------------------------------------
def dft_mats_1d(n, K):
    """Forward F[k, x] = exp(-2 pi i k x / n) and inverse E[x, k] such that the
    inverse of the truncated real spectrum is Re(E @ What) (k = 0..K-1 < n/2)."""
    x = np.arange(n)
    k = np.arange(K)
    F = np.exp(-2j * np.pi * np.outer(k, x) / n)
    c = np.where(k == 0, 1.0, 2.0)
    E = (c[None, :] / n) * np.exp(2j * np.pi * np.outer(x, k) / n)
    return F, E


def spectral1d_forward(v, Rr, Ri, quant=_id):
    """v: (B, n, C); R = Rr + i Ri: (K, C, O).  Returns u (B, n, O), cache."""
    B, n, C = v.shape
    K = Rr.shape[0]
    F, E = dft_mats_1d(n, K)
    Vh = np.einsum("kx,bxc->bkc", F, quant(v))
    R = quant(Rr) + 1j * quant(Ri)
    Vq = quant(Vh.real) + 1j * quant(Vh.imag)
    Wh = np.einsum("bkc,kco->bko", Vq, R)
    u = np.einsum("xk,bko->bxo", E, Wh).real
    return u, (v, Vq, R, F, E)


def spectral1d_backward(cache, du, quant=_id):
    v, Vq, R, F, E = cache
    gW = np.einsum("xk,bxo->bko", np.conj(E), du)       # dRe + i dIm of What
    gR = np.einsum("bkc,bko->kco", np.conj(Vq), gW)
    gV = np.einsum("bko,kco->bkc", gW, np.conj(R))
    dv = np.einsum("kx,bkc->bxc", np.conj(F), gV).real
    return dv, gR.real, gR.imag


def fno1d_forward(params, S, xcoord, quant=_id, n_layers=4):
    """S: (B, n) source; xcoord: (n,) normalised coordinate.  Returns (B, n)."""
    B, n = S.shape
    inp = np.stack([S, np.broadcast_to(xcoord, (B, n))], axis=-1)   # (B, n, 2)
    cache = {"inp": inp}
    v = quant(inp) @ quant(params["lift.W"]).T + params["lift.b"]
    cache["v0"] = v
    for l in range(n_layers):
        us, sc = spectral1d_forward(v, params["spec%d.re" % l], params["spec%d.im" % l], quant)
        z = us + quant(v) @ quant(params["pw%d.W" % l]).T + params["pw%d.b" % l]
        cache["spec%d" % l] = sc
        cache["z%d" % l] = z
        v = np.maximum(z, 0.0)
        cache["v%d" % (l + 1)] = v
    h = quant(v) @ quant(params["proj1.W"]).T + params["proj1.b"]
    cache["h"] = h
    a = np.maximum(h, 0.0)
    out = (quant(a) @ quant(params["proj2.W"]).T + params["proj2.b"])[..., 0]
    cache["a"] = a
    return out, cache


def fno1d_backward(params, cache, dout, quant=_id, n_layers=4):
    grads = {}
    g = dout[..., None]                                  # (B, n, 1)
    a = cache["a"]
    grads["proj2.W"] = np.einsum("bxo,bxi->oi", quant(g), quant(a))
    grads["proj2.b"] = g.sum(axis=(0, 1))
    g = quant(g) @ quant(params["proj2.W"])
    g = g * (cache["h"] > 0)
    v = cache["v%d" % n_layers]
    grads["proj1.W"] = np.einsum("bxo,bxi->oi", quant(g), quant(v))
    grads["proj1.b"] = g.sum(axis=(0, 1))
    g = quant(g) @ quant(params["proj1.W"])
    for l in range(n_layers - 1, -1, -1):
        g = g * (cache["z%d" % l] > 0)
        v = cache["v%d" % l]
        grads["pw%d.W" % l] = np.einsum("bxo,bxi->oi", quant(g), quant(v))
        grads["pw%d.b" % l] = g.sum(axis=(0, 1))
        dv_pw = quant(g) @ quant(params["pw%d.W" % l])
        dv_sp, gr, gi = spectral1d_backward(cache["spec%d" % l], g, quant)
        grads["spec%d.re" % l], grads["spec%d.im" % l] = gr, gi
        g = dv_pw + dv_sp
    inp = cache["inp"]
    grads["lift.W"] = np.einsum("bxo,bxi->oi", quant(g), quant(inp))
    grads["lift.b"] = g.sum(axis=(0, 1))
    return grads


# ----------------------------------------------------------------------------
# FNO 2D
# ----------------------------------------------------------------------------
def dft_mats_2d(ny, nx, m1, m2):
    """Row transform over k_y in {0..m1-1} U {ny-m1..ny-1} and column transform
    over k_x in {0..m2-1}; inverse weights c = 1 for k_x = 0 else 2."""
    ky = np.concatenate([np.arange(m1), np.arange(ny - m1, ny)])
    kx = np.arange(m2)
    y, x = np.arange(ny), np.arange(nx)
    Fy = np.exp(-2j * np.pi * np.outer(ky, y) / ny)          # (2m1, ny)
    Fx = np.exp(-2j * np.pi * np.outer(kx, x) / nx)          # (m2, nx)
    Ey = np.exp(2j * np.pi * np.outer(y, ky) / ny) / ny      # (ny, 2m1)
    c = np.where(kx == 0, 1.0, 2.0)
    Ex = (c[None, :] / nx) * np.exp(2j * np.pi * np.outer(x, kx) / nx)   # (nx, m2)
    return Fy, Fx, Ey, Ex


def spectral2d_forward(v, R1r, R1i, R2r, R2i, quant=_id):
    """v: (B, ny, nx, C); R1, R2: (m1, m2, C, O).  Returns u (B, ny, nx, O)."""
    B, ny, nx, C = v.shape
    m1, m2 = R1r.shape[:2]
    Fy, Fx, Ey, Ex = dft_mats_2d(ny, nx, m1, m2)
    Vh = np.einsum("ky,lx,byxc->bklc", Fy, Fx, quant(v), optimize=True)      # (B, 2m1, m2, C)
    Vq = quant(Vh.real) + 1j * quant(Vh.imag)
    R = np.concatenate([quant(R1r) + 1j * quant(R1i), quant(R2r) + 1j * quant(R2i)], axis=0)
    Wh = np.einsum("bklc,klco->bklo", Vq, R)
    u = np.einsum("yk,xl,bklo->byxo", Ey, Ex, Wh, optimize=True).real
    return u, (Vq, R, Fy, Fx, Ey, Ex, m1)


def spectral2d_backward(cache, du, quant=_id):
    Vq, R, Fy, Fx, Ey, Ex, m1 = cache
    gW = np.einsum("yk,xl,byxo->bklo", np.conj(Ey), np.conj(Ex), du, optimize=True)
    gR = np.einsum("bklc,bklo->klco", np.conj(Vq), gW)
    gV = np.einsum("bklo,klco->bklc", gW, np.conj(R))
    dv = np.einsum("ky,lx,bklc->byxc", np.conj(Fy), np.conj(Fx), gV, optimize=True).real
    return dv, (gR[:m1].real, gR[:m1].imag, gR[m1:].real, gR[m1:].imag)


def fno2d_forward(params, S, ycoord, xcoord, quant=_id, n_layers=4):
    """S: (B, ny, nx); coordinates (ny,), (nx,).  Returns (B, ny, nx)."""
    B, ny, nx = S.shape
    Yc = np.broadcast_to(ycoord[:, None], (ny, nx))
    Xc = np.broadcast_to(xcoord[None, :], (ny, nx))
    inp = np.stack([S, np.broadcast_to(Xc, S.shape), np.broadcast_to(Yc, S.shape)], axis=-1)
    cache = {"inp": inp}
    v = quant(inp) @ quant(params["lift.W"]).T + params["lift.b"]
    for l in range(n_layers):
        us, sc = spectral2d_forward(v, params["spec%d.re1" % l], params["spec%d.im1" % l],
                                    params["spec%d.re2" % l], params["spec%d.im2" % l], quant)
        z = us + quant(v) @ quant(params["pw%d.W" % l]).T + params["pw%d.b" % l]
        cache["v%d" % l] = v
        cache["spec%d" % l] = sc
        cache["z%d" % l] = z
        v = np.maximum(z, 0.0)
    cache["v%d" % n_layers] = v
    h = quant(v) @ quant(params["proj1.W"]).T + params["proj1.b"]
    a = np.maximum(h, 0.0)
    cache["h"], cache["a"] = h, a
    out = (quant(a) @ quant(params["proj2.W"]).T + params["proj2.b"])[..., 0]
    return out, cache


def fno2d_backward(params, cache, dout, quant=_id, n_layers=4):
    grads = {}
    g = dout[..., None]
    a = cache["a"]
    grads["proj2.W"] = np.einsum("byxo,byxi->oi", quant(g), quant(a))
    grads["proj2.b"] = g.sum(axis=(0, 1, 2))
    g = quant(g) @ quant(params["proj2.W"])
    g = g * (cache["h"] > 0)
    v = cache["v%d" % n_layers]
    grads["proj1.W"] = np.einsum("byxo,byxi->oi", quant(g), quant(v))
    grads["proj1.b"] = g.sum(axis=(0, 1, 2))
    g = quant(g) @ quant(params["proj1.W"])
    for l in range(n_layers - 1, -1, -1):
        g = g * (cache["z%d" % l] > 0)
        v = cache["v%d" % l]
        grads["pw%d.W" % l] = np.einsum("byxo,byxi->oi", quant(g), quant(v))
        grads["pw%d.b" % l] = g.sum(axis=(0, 1, 2))
        dv_pw = quant(g) @ quant(params["pw%d.W" % l])
        dv_sp, (r1, i1, r2, i2) = spectral2d_backward(cache["spec%d" % l], g, quant)
        grads["spec%d.re1" % l], grads["spec%d.im1" % l] = r1, i1
        grads["spec%d.re2" % l], grads["spec%d.im2" % l] = r2, i2
        g = dv_pw + dv_sp
    inp = cache["inp"]
    grads["lift.W"] = np.einsum("byxo,byxi->oi", quant(g), quant(inp))
    grads["lift.b"] = g.sum(axis=(0, 1, 2))
    return grads


# ----------------------------------------------------------------------------
# loss and optimiser
# ----------------------------------------------------------------------------
def mse(out, target):
    """Mean squared error over all entries and its gradient (Table A1)."""
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), in place; t is the 1-based step count."""
    for k in params:
        g = grads[k]
        m[k] = b1 * m[k] + (1 - b1) * g
        v[k] = b2 * v[k] + (1 - b2) * g * g
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


def param_count(params):
    return int(sum(np.asarray(p).size for p in params.values()))
