"""FP64 numpy oracle of the warm-start network -- TEST INFRASTRUCTURE ONLY.

The same encoder-decoder as the CUDA path (3D convolutions 1-16-32-64-32-16
with 3^3 kernels and zero padding, 2^3 average pooling, 2^3 nearest
upsampling, additive skips, ReLU, a 1^3 head to 2 outputs), written as plain
numpy in FP64.  With `bf=True` it rounds to BF16 (round-to-nearest-even)
exactly where the CUDA path stores BF16 (weights of the four inner
convolutions, stored activations, the pre-activation gradients fed to those
convolutions), so both sides take the same ReLU decisions; with `bf=False` it
is the plain FP64 network, pinned by finite differences and by
scipy.ndimage.correlate.
"""
import numpy as np

LAYERS = [(1, 16, 27), (16, 32, 27), (32, 64, 27), (64, 32, 27), (32, 16, 27), (16, 2, 1)]


def n_params():
    return sum(t * ci * co + co for ci, co, t in LAYERS)


def unpack(params):
    """[(W [taps, ci, co], b [co])] from the flat parameter vector."""
    params = np.asarray(params, np.float64)
    out, o = [], 0
    for ci, co, t in LAYERS:
        w = params[o:o + t * ci * co].reshape(t, ci, co)
        o += t * ci * co
        b = params[o:o + co]
        o += co
        out.append((w, b))
    return out


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    x32 = np.ascontiguousarray(np.asarray(x, np.float32))
    u = x32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def taps():
    """Offsets (dx, dy, dz) in tap order: tap = 9 (dz+1) + 3 (dy+1) + (dx+1)."""
    return [(t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1) for t in range(27)]


def conv3(x, w):
    """y[z,y,x,co] = sum_tap sum_ci x[z+dz, y+dy, x+dx, ci] w[tap, ci, co] (zero padding).
    x: [n,n,n,ci] channels-last."""
    n = x.shape[0]
    xp = np.zeros((n + 2, n + 2, n + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    y = np.zeros((n, n, n, w.shape[2]))
    for t, (dx, dy, dz) in enumerate(taps()):
        sl = xp[1 + dz:1 + dz + n, 1 + dy:1 + dy + n, 1 + dx:1 + dx + n]
        y += sl @ w[t]
    return y


def conv3_wgrad(x, g):
    """d/dw of sum(g * conv3(x, w)): [27, ci, co]."""
    n = x.shape[0]
    xp = np.zeros((n + 2, n + 2, n + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    out = np.zeros((27, x.shape[3], g.shape[3]))
    for t, (dx, dy, dz) in enumerate(taps()):
        sl = xp[1 + dz:1 + dz + n, 1 + dy:1 + dy + n, 1 + dx:1 + dx + n]
        out[t] = sl.reshape(-1, x.shape[3]).T @ g.reshape(-1, g.shape[3])
    return out


def conv3_dgrad(g, w):
    """d/dx of sum(g * conv3(x, w)): [n,n,n,ci]."""
    n = g.shape[0]
    out = np.zeros((n + 2, n + 2, n + 2, w.shape[1]))
    for t, (dx, dy, dz) in enumerate(taps()):
        out[1 + dz:1 + dz + n, 1 + dy:1 + dy + n, 1 + dx:1 + dx + n] += g @ w[t].T
    return out[1:-1, 1:-1, 1:-1]


def pool(x):
    n = x.shape[0] // 2
    return x.reshape(n, 2, n, 2, n, 2, -1).mean(axis=(1, 3, 5))


def pool_T(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_T(g):
    n = g.shape[0] // 2
    return g.reshape(n, 2, n, 2, n, 2, -1).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, x, bf=True):
    """x: [n,n,n] input; returns (y [n,n,n,2], cache)."""
    q = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    P = unpack(params)
    x = np.asarray(x, np.float64)[..., None]
    W = [P[0][0]] + [q(P[l][0]) for l in range(1, 5)] + [P[5][0]]
    b = [P[l][1] for l in range(6)]
    a1 = q(relu(conv3(x, W[0]) + b[0]))
    p1 = q(pool(a1))
    a2 = q(relu(conv3(p1, W[1]) + b[1]))
    p2 = q(pool(a2))
    a3 = q(relu(conv3(p2, W[2]) + b[2]))
    u2 = up(a3)
    a4 = q(relu(conv3(u2, W[3]) + b[3] + a2))
    u1 = up(a4)
    a5 = q(relu(conv3(u1, W[4]) + b[4] + a1))
    y = a5 @ W[5][0] + b[5]
    return y, dict(x=x, W=W, a1=a1, p1=p1, a2=a2, p2=p2, a3=a3, u2=u2, a4=a4, u1=u1, a5=a5)


def backward(params, x, gy, bf=True):
    """Gradient of sum(gy * y) w.r.t. the flat parameters."""
    q = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    _, c = forward(params, x, bf)
    W = c["W"]
    gy = np.asarray(gy, np.float64)
    grads = []
    # head
    dW5 = c["a5"].reshape(-1, 16).T @ gy.reshape(-1, 2)
    db5 = gy.reshape(-1, 2).sum(0)
    ga5 = gy @ W[5][0].T
    gz5 = (c["a5"] > 0) * ga5
    dW4 = conv3_wgrad(c["u1"], q(gz5)); db4 = gz5.reshape(-1, 16).sum(0)
    gu1 = conv3_dgrad(q(gz5), W[4])
    gz4 = (c["a4"] > 0) * up_T(gu1)
    dW3 = conv3_wgrad(c["u2"], q(gz4)); db3 = gz4.reshape(-1, 32).sum(0)
    gu2 = conv3_dgrad(q(gz4), W[3])
    gz3 = (c["a3"] > 0) * up_T(gu2)
    dW2 = conv3_wgrad(c["p2"], q(gz3)); db2 = gz3.reshape(-1, 64).sum(0)
    gp2 = conv3_dgrad(q(gz3), W[2])
    gz2 = (c["a2"] > 0) * (gz4 + pool_T(gp2))
    dW1 = conv3_wgrad(c["p1"], q(gz2)); db1 = gz2.reshape(-1, 32).sum(0)
    gp1 = conv3_dgrad(q(gz2), W[1])
    gz1 = (c["a1"] > 0) * (gz5 + pool_T(gp1))
    dW0 = conv3_wgrad(c["x"], gz1); db0 = gz1.reshape(-1, 16).sum(0)
    for dw, db in ((dW0, db0), (dW1, db1), (dW2, db2), (dW3, db3), (dW4, db4), (dW5[None], db5)):
        grads.append(dw.reshape(-1)); grads.append(db)
    return np.concatenate(grads)


def ramlak_filter(sino, pu, beam, dsd=0.0, pv=1.0):
    """Cosine-weighted (cone) Ram-Lak filtering of every detector row by direct
    convolution: h(0) = 1/(4 p^2), h(odd k) = -1/(pi k p)^2, h(even k) = 0,
    times the pitch p."""
    sino = np.asarray(sino, np.float64)
    V, nv, nu = sino.shape
    u = (np.arange(nu) - 0.5 * (nu - 1)) * pu
    v = (np.arange(nv) - 0.5 * (nv - 1)) * pv
    if beam == 1:
        w = dsd / np.sqrt(dsd ** 2 + u[None, :] ** 2 + v[:, None] ** 2)
    else:
        w = np.ones((nv, nu))
    k = np.arange(-(nu - 1), nu)
    kk = np.where(k == 0, 1, k).astype(np.float64)
    h = np.where(k == 0, 1.0 / (4 * pu * pu), np.where(k % 2 != 0, -1.0 / (np.pi * kk * pu) ** 2, 0.0))
    out = np.zeros_like(sino)
    for i in range(nu):
        out[:, :, i] = ((sino * w[None]) * h[(i - np.arange(nu)) + nu - 1][None, None, :]).sum(-1) * pu
    return out
