"""FP64 oracle of the learned CG preconditioner (test infrastructure only).

The paper names the missing piece of time-domain ESI: an efficient preconditioner that
reduces the number of inner CG iterations (Conclusion; the storage section calls good
preconditioning a bottleneck).  The preconditioner built here is

    z = s + up2(U_theta(pack(s))),       s = r / (beta B^2)

i.e. the diagonal preconditioner of the ESI normal operator (its beta B^T B part) plus a
learned correction.  pack() groups G = 16 consecutive time samples of s as channels and
averages 2 x 2 cells; U_theta is a 4-level U-Net with 32 channels (3 x 3 convolutions,
zero padding, ReLU, 2 x 2 average pooling with zero fill at odd edges, nearest
upsampling with skip additions); up2 repeats each coarse cell over its 2 x 2 block.
The network is a learned object: its parity is unpinned; the CG residual judges it.
The building blocks (convolution, pooling, upsampling, the backward pass, the loss,
Adam) are plain definitions and are pinned by the CPU tests.

Layouts: images channels-last, x[img][h][w][c]; weights W[dy][dx][ci][co], biases b[co].
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

G = 16          # time samples per image (channels of the network input / output)
C = 32          # hidden channels
LEVELS = 4

# layer list: (name, cin, cout, relu)
LAYERS = [("enc1", G, C, True), ("enc2", C, C, True), ("enc3", C, C, True), ("bott", C, C, True),
          ("dec3", C, C, True), ("dec2", C, C, True), ("dec1", C, G, False)]


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n,h,w,co] = b[co] + sum_{dy,dx,ci} x[n, h+dy-1, w+dx-1, ci] W[dy,dx,ci,co],
    zero outside the image."""
    n, H, Wd, ci = x.shape
    co = W.shape[3]
    xp = np.zeros((n, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((n, H, Wd, co)) + b
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nhwc,cd->nhwd", xp[:, dy:dy + H, dx:dx + Wd, :], W[dy, dx])
    return y


def conv3x3_backward(x: np.ndarray, W: np.ndarray, gy: np.ndarray
                     ) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Gradients of sum(gy * conv3x3(x, W, b)) with respect to x, W and b."""
    n, H, Wd, ci = x.shape
    xp = np.zeros((n, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gW[dy, dx] = np.einsum("nhwc,nhwd->cd", xp[:, dy:dy + H, dx:dx + Wd, :], gy)
            gxp[:, dy:dy + H, dx:dx + Wd, :] += np.einsum("nhwd,cd->nhwc", gy, W[dy, dx])
    gb = gy.sum(axis=(0, 1, 2))
    return gxp[:, 1:-1, 1:-1, :], gW, gb


def pool2(x: np.ndarray) -> np.ndarray:
    """0.25 * sum of each 2 x 2 block; cells beyond an odd edge count as zero."""
    n, H, Wd, c = x.shape
    Ho, Wo = (H + 1) // 2, (Wd + 1) // 2
    xp = np.zeros((n, 2 * Ho, 2 * Wo, c))
    xp[:, :H, :Wd, :] = x
    return 0.25 * (xp[:, 0::2, 0::2] + xp[:, 1::2, 0::2] + xp[:, 0::2, 1::2] + xp[:, 1::2, 1::2])


def pool2_backward(gy: np.ndarray, H: int, Wd: int) -> np.ndarray:
    g = 0.25 * np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2)
    return g[:, :H, :Wd, :]


def up2(x: np.ndarray, H: int, Wd: int) -> np.ndarray:
    """Nearest upsampling: out[h, w] = x[h // 2, w // 2], cropped to H x Wd."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)[:, :H, :Wd, :]


def up2_backward(gy: np.ndarray, Hc: int, Wc: int) -> np.ndarray:
    n, H, Wd, c = gy.shape
    g = np.zeros((n, 2 * Hc, 2 * Wc, c))
    g[:, :H, :Wd, :] = gy
    return g[:, 0::2, 0::2] + g[:, 1::2, 0::2] + g[:, 0::2, 1::2] + g[:, 1::2, 1::2]


def init_params(seed: int, scale: float = 1.0) -> Dict[str, np.ndarray]:
    """He-style random weights (std sqrt(2 / (9 cin))) times `scale`; zero biases; the last
    layer starts at zero so that the untrained preconditioner is the diagonal one."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co, _ in LAYERS:
        std = scale * math.sqrt(2.0 / (9 * ci))
        p[name + ".W"] = rng.standard_normal((3, 3, ci, co)) * std
        p[name + ".b"] = np.zeros(co)
    p["dec1.W"][:] = 0.0
    return p


def unet_forward(x: np.ndarray, p: Dict[str, np.ndarray], store=None) -> Tuple[np.ndarray, Dict]:
    """4-level U-Net; returns the output and the activations needed by the backward.
    ``store`` (optional) maps every stored hidden activation (conv outputs, pooled and
    upsampled-plus-skip tensors) to the values a reduced-precision implementation keeps;
    the default keeps them exactly."""
    st = store if store is not None else (lambda t: t)
    a = {"x": x}

    def layer(name, inp, relu):
        pre = conv3x3(inp, p[name + ".W"], p[name + ".b"])
        a[name + ".in"] = inp
        a[name + ".pre"] = pre
        return st(np.maximum(pre, 0.0)) if relu else pre
    e1 = layer("enc1", x, True)
    e2 = layer("enc2", st(pool2(e1)), True)
    e3 = layer("enc3", st(pool2(e2)), True)
    bt = layer("bott", st(pool2(e3)), True)
    d3 = layer("dec3", st(up2(bt, *e3.shape[1:3]) + e3), True)
    d2 = layer("dec2", st(up2(d3, *e2.shape[1:3]) + e2), True)
    y = layer("dec1", st(up2(d2, *e1.shape[1:3]) + e1), False)
    a.update(e1=e1, e2=e2, e3=e3, bt=bt, d3=d3, d2=d2)
    return y, a


def normalized_forward(x: np.ndarray, p: Dict[str, np.ndarray], store=None
                       ) -> Tuple[np.ndarray, Dict, np.ndarray]:
    """y_i = rho_i U(x_i / rho_i), rho_i the root-mean-square of image i (y_i = 0 when
    rho_i = 0): positively homogeneous in x, as a preconditioner has to be."""
    st = store if store is not None else (lambda t: t)
    rho = np.sqrt(np.mean(x.reshape(x.shape[0], -1) ** 2, axis=1))
    safe = np.where(rho > 0, rho, 1.0)
    xn = st(np.where(rho[:, None, None, None] > 0, x / safe[:, None, None, None], 0.0))
    y, a = unet_forward(xn, p, store)
    return y * rho[:, None, None, None], a, rho


def unet_backward(gy: np.ndarray, p: Dict[str, np.ndarray], a: Dict) -> Tuple[np.ndarray, Dict]:
    """Gradients of sum(gy * y) with respect to the input and every parameter."""
    g = {}

    def layer_back(name, gout, relu):
        if relu:
            gout = gout * (a[name + ".pre"] > 0)
        gin, gW, gb = conv3x3_backward(a[name + ".in"], p[name + ".W"], gout)
        g[name + ".W"], g[name + ".b"] = gW, gb
        return gin
    e1, e2, e3, bt, d2, d3 = a["e1"], a["e2"], a["e3"], a["bt"], a["d2"], a["d3"]
    gin = layer_back("dec1", gy, False)               # input of dec1 = up(d2) + e1
    g_e1 = gin.copy()
    g_d2 = up2_backward(gin, *d2.shape[1:3])
    gin = layer_back("dec2", g_d2, True)              # input = up(d3) + e2
    g_e2 = gin.copy()
    g_d3 = up2_backward(gin, *d3.shape[1:3])
    gin = layer_back("dec3", g_d3, True)              # input = up(bt) + e3
    g_e3 = gin.copy()
    g_bt = up2_backward(gin, *bt.shape[1:3])
    gin = layer_back("bott", g_bt, True)              # input = pool(e3)
    g_e3 += pool2_backward(gin, *e3.shape[1:3])
    gin = layer_back("enc3", g_e3, True)              # input = pool(e2)
    g_e2 += pool2_backward(gin, *e2.shape[1:3])
    gin = layer_back("enc2", g_e2, True)              # input = pool(e1)
    g_e1 += pool2_backward(gin, *e1.shape[1:3])
    gx = layer_back("enc1", g_e1, True)
    return gx, g


def pack(s: np.ndarray) -> np.ndarray:
    """s[t][z][x] (one shot, nt a multiple of G) -> images [nt/G][ceil(z/2)][ceil(x/2)][G]:
    channel c of image g is time sample G g + c, 2 x 2 averaged (zero fill at odd edges)."""
    nt, nz, nx = s.shape
    img = s.reshape(nt // G, G, nz, nx).transpose(0, 2, 3, 1)
    return pool2(img)


def unpack(s: np.ndarray, y: np.ndarray) -> np.ndarray:
    """z[t][z][x] = s[t][z][x] + y[t // G][z // 2][x // 2][t % G]."""
    nt, nz, nx = s.shape
    u = up2(y, nz, nx)                                  # [nt/G][nz][nx][G]
    return s + u.transpose(0, 3, 1, 2).reshape(nt, nz, nx)


def precondition(r: np.ndarray, D: np.ndarray, p: Dict[str, np.ndarray]) -> np.ndarray:
    """z = s + up2(rho U(pack(s) / rho)), s = D * r (D = 1 / (beta B^2) per cell), rho the
    per-image root-mean-square of pack(s)."""
    s = r * D[None]
    y, _, _ = normalized_forward(pack(s), p)
    return unpack(s, y)


def param_vector(p: Dict[str, np.ndarray]) -> np.ndarray:
    """Flat parameter vector in the library's order: per layer W[3][3][cin][cout], b[cout]."""
    return np.concatenate([np.concatenate([p[n + ".W"].ravel(), p[n + ".b"].ravel()])
                           for n, _, _, _ in LAYERS])


def params_from_vector(v: np.ndarray) -> Dict[str, np.ndarray]:
    p, o = {}, 0
    for n, ci, co, _ in LAYERS:
        k = 9 * ci * co
        p[n + ".W"] = np.asarray(v[o:o + k], dtype=np.float64).reshape(3, 3, ci, co)
        p[n + ".b"] = np.asarray(v[o + k:o + k + co], dtype=np.float64)
        o += k + co
    return p


def batch_loss_and_grad(x: np.ndarray, e: np.ndarray, p: Dict[str, np.ndarray], store=None
                        ) -> Tuple[float, Dict[str, np.ndarray]]:
    """Training objective on a batch: mean_i cosine_loss(x_i + y_i, e_i) with the normalised
    network y = rho U(x / rho), and its gradient with respect to every parameter."""
    y, a, rho = normalized_forward(x, p, store)
    n = x.shape[0]
    gy = np.zeros_like(y)
    loss = 0.0
    for i in range(n):
        z = x[i] + y[i]
        loss += cosine_loss(z, e[i])
        gy[i] = cosine_loss_grad(z, e[i]) / n * rho[i]   # y = rho U(x / rho)
    _, g = unet_backward(gy, p, a)
    return loss / n, g


def cosine_loss(z: np.ndarray, e: np.ndarray) -> float:
    """1 - <z, e>^2 / (|z|^2 |e|^2): scale-free misfit of the preconditioned direction."""
    ze, zz, ee = float(np.sum(z * e)), float(np.sum(z * z)), float(np.sum(e * e))
    return 1.0 - ze * ze / (zz * ee)


def cosine_loss_grad(z: np.ndarray, e: np.ndarray) -> np.ndarray:
    ze, zz, ee = float(np.sum(z * e)), float(np.sum(z * z)), float(np.sum(e * e))
    return -(2.0 * ze / (zz * ee)) * e + (2.0 * ze * ze / (zz * zz * ee)) * z


def adam_step(p: Dict, g: Dict, m: Dict, v: Dict, t: int, lr: float, b1: float = 0.9,
              b2: float = 0.999, eps: float = 1e-8) -> None:
    """Adam (Kingma & Ba 2015) with bias correction, in place."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
