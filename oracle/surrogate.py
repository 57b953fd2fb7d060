"""FP64 reference of the learned orbital surrogate (test infrastructure only).

The surrogate replaces the B-spline table by a small learned function of
the position: a periodic multiresolution hashed grid of features followed by
a multilayer perceptron whose outputs are the N orbitals.  It aims at the
memory footprint the paper attacks (arXiv 1708.02645, Sec. 6.3 and the
memory results of Sec. 6.4, up to 3.8x smaller); the B-spline stays the
arbiter of its error.  The paper has no such surrogate, so this file fixes the function
the GPU kernels must compute:

* levels l = 0..L-1 with resolutions R_l = floor(R_min * b^l), b =
  (R_max / R_min)^(1 / (L - 1)); level l's table has T entries of F
  features; corner (i, j, k) of a level (taken modulo R_l: the function is
  periodic on the unit cube) is stored densely at (i R_l + j) R_l + k when
  R_l^3 <= T, else at the spatial hash (i ^ 2654435761 j ^ 805459861 k) mod T;
* each level interpolates its 8 corners with the C2 weights s(t) = t^3 (6 t^2
  - 15 t + 10) and 1 - s(t) per axis, so values, gradients and Laplacians of
  the features exist everywhere;
* the L F features feed a perceptron with softplus hidden layers (smooth,
  so that the Laplacian of the output does not vanish) and a linear output
  layer of N orbitals.

Every quantity carries five channels through the network, (value, d/dx,
d/dy, d/dz, Laplacian): a linear layer maps each channel with the same
weights (the bias only enters the value), and h = softplus(z) maps them as
h = sp(z), dh = sp'(z) dz, lap h = sp''(z) |dz|^2 + sp'(z) lap z.  The
output channels are directly the surrogate's V, G and L.

Training minimises sum_c w_c mean((out_c - target_c)^2) over the channels
(w_c fixes the weight of V, of each gradient component and of L); grads()
is the hand-derived backward of that loss, pinned by finite differences in
tests/test_surrogate_reference.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PRIME_Y = 2654435761
PRIME_Z = 805459861


@dataclass
class SurrogateSpec:
    levels: int = 16
    log2_table: int = 19
    features: int = 2
    r_min: int = 16
    r_max: int = 512
    hidden: int = 128
    layers: int = 3
    N: int = 384

    @property
    def table(self) -> int:
        return 1 << self.log2_table

    def resolutions(self):
        if self.levels == 1:
            return [self.r_min]
        b = (self.r_max / self.r_min) ** (1.0 / (self.levels - 1))
        return [int(math.floor(self.r_min * b ** l + 1e-9)) for l in range(self.levels)]

    def widths(self):
        return [self.levels * self.features] + [self.hidden] * self.layers + [self.N]


@dataclass
class SurrogateParams:
    spec: SurrogateSpec
    grid: np.ndarray            # [levels, T, F]
    W: list = field(default_factory=list)    # W[l]: [out, in]
    b: list = field(default_factory=list)    # b[l]: [out]


def corner_slot(R: int, T: int, i, j, k):
    """Table slot of corner (i, j, k) (already reduced modulo R)."""
    i, j, k = (np.asarray(v, dtype=np.int64) for v in (i, j, k))
    if R * R * R <= T:
        return (i * R + j) * R + k
    h = (i.astype(np.uint64) ^ (j.astype(np.uint64) * np.uint64(PRIME_Y))
         ^ (k.astype(np.uint64) * np.uint64(PRIME_Z)))
    return (h & np.uint64(T - 1)).astype(np.int64)


def smooth(t):
    """s(t), s'(t), s''(t) of the C2 interpolation weight."""
    s = t * t * t * (t * (6.0 * t - 15.0) + 10.0)
    ds = 30.0 * t * t * (t - 1.0) * (t - 1.0)
    d2s = 60.0 * t * (t - 1.0) * (2.0 * t - 1.0)
    return s, ds, d2s


def encode(params: SurrogateParams, pos):
    """Features with channels: [P, 5, levels * F]; also returns, per level,
    the corner slots and the 5-channel corner weights for the backward."""
    spec = params.spec
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    P = pos.shape[0]
    out = np.zeros((P, 5, spec.levels * spec.features))
    cache = []
    for l, R in enumerate(spec.resolutions()):
        u = pos * R
        fl = np.floor(u)
        t = u - fl
        cell = np.mod(fl.astype(np.int64), R)
        s, ds, d2s = smooth(t)                       # [P, 3]
        # per axis: weight of corner bit 0 / 1, first and second derivative (d/dr)
        w = [np.stack([1.0 - s[:, d], s[:, d]], 1) for d in range(3)]
        dw = [np.stack([-ds[:, d], ds[:, d]], 1) * R for d in range(3)]
        d2w = [np.stack([-d2s[:, d], d2s[:, d]], 1) * R * R for d in range(3)]
        slots = np.zeros((P, 8), dtype=np.int64)
        cw = np.zeros((P, 5, 8))
        for c in range(8):
            bx, by, bz = (c >> 2) & 1, (c >> 1) & 1, c & 1
            slots[:, c] = corner_slot(R, spec.table, (cell[:, 0] + bx) % R, (cell[:, 1] + by) % R,
                                      (cell[:, 2] + bz) % R)
            wx, wy, wz = w[0][:, bx], w[1][:, by], w[2][:, bz]
            cw[:, 0, c] = wx * wy * wz
            cw[:, 1, c] = dw[0][:, bx] * wy * wz
            cw[:, 2, c] = wx * dw[1][:, by] * wz
            cw[:, 3, c] = wx * wy * dw[2][:, bz]
            cw[:, 4, c] = (d2w[0][:, bx] * wy * wz + wx * d2w[1][:, by] * wz
                           + wx * wy * d2w[2][:, bz])
        theta = params.grid[l][slots]                # [P, 8, F]
        out[:, :, l * spec.features:(l + 1) * spec.features] = np.einsum("pcq,pqf->pcf", cw, theta)
        cache.append((slots, cw))
    return out, cache


def softplus(z):
    """sp(z) and its first three derivatives (stable form)."""
    sp = np.logaddexp(0.0, z)
    sg = 0.5 * (1.0 + np.tanh(0.5 * z))              # sigmoid
    return sp, sg, sg * (1.0 - sg), sg * (1.0 - sg) * (1.0 - 2.0 * sg)


def round_bf16(x):
    """Round to the nearest bfloat16 (8 significant bits, ties to even)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                     # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def round_fp16(x):
    """Round to the nearest IEEE binary16 (ties to even, subnormals kept)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def quantised(params: SurrogateParams) -> SurrogateParams:
    """The inference copy: grid in binary16, weights in bfloat16, biases
    as they are."""
    return SurrogateParams(params.spec, round_fp16(params.grid), [round_bf16(w) for w in params.W],
                           [np.array(b) for b in params.b])


def forward(params: SurrogateParams, pos, act_round=None, gemm_round=None):
    """Surrogate outputs [P, 5, N] (V, Gx, Gy, Gz, L) and the intermediates.
    act_round, if given, is applied to every layer's input (all channels):
    the inference precision rounds activations to bfloat16 there.
    gemm_round, if given, is applied to both operands of every layer's
    product (input and weights), as the tensor-core training reads them; the
    stored intermediates stay unrounded."""
    h, enc_cache = encode(params, pos)
    acts = [h]
    pre = []
    nl = len(params.W)
    for l in range(nl):
        if act_round is not None:
            h = act_round(h)
        if gemm_round is not None:
            z = np.einsum("pci,oi->pco", gemm_round(h), gemm_round(params.W[l]))
        else:
            z = np.einsum("pci,oi->pco", h, params.W[l])
        z[:, 0, :] += params.b[l]
        pre.append(z)
        if l == nl - 1:
            h = z
        else:
            sp, d1, d2, _ = softplus(z[:, 0, :])
            g2 = (z[:, 1:4, :] ** 2).sum(1)
            h = np.empty_like(z)
            h[:, 0] = sp
            h[:, 1:4] = d1[:, None, :] * z[:, 1:4]
            h[:, 4] = d2 * g2 + d1 * z[:, 4]
        acts.append(h)
    return h, (acts, pre, enc_cache)


def loss(out, target, wch):
    """sum_c w_c mean over (positions, orbitals) of (out_c - target_c)^2."""
    d = np.asarray(out) - np.asarray(target)
    return float(sum(wch[c] * np.mean(d[:, c] ** 2) for c in range(5)))


def grads(params: SurrogateParams, pos, target, wch, gemm_round=None):
    """Loss and its gradients with respect to the grid table, W and b.
    gemm_round, if given, rounds both operands of every product (forward,
    weight gradient, data gradient): the tensor-core training reading."""
    R = gemm_round if gemm_round is not None else (lambda x: x)
    out, (acts, pre, enc_cache) = forward(params, pos, gemm_round=gemm_round)
    P, _, N = out.shape
    g = np.zeros_like(out)
    for c in range(5):
        g[:, c] = 2.0 * wch[c] * (out[:, c] - target[:, c]) / (P * N)
    gW, gb = [None] * len(params.W), [None] * len(params.W)
    nl = len(params.W)
    for l in range(nl - 1, -1, -1):
        if l == nl - 1:
            gz = g
        else:
            z = pre[l]
            _, d1, d2, d3 = softplus(z[:, 0, :])
            zd = z[:, 1:4, :]
            g2 = (zd ** 2).sum(1)
            gz = np.empty_like(z)
            gz[:, 0] = (g[:, 0] * d1 + (g[:, 1:4] * zd).sum(1) * d2
                        + g[:, 4] * (d3 * g2 + d2 * z[:, 4]))
            gz[:, 1:4] = g[:, 1:4] * d1[:, None, :] + 2.0 * (g[:, 4] * d2)[:, None, :] * zd
            gz[:, 4] = g[:, 4] * d1
        gW[l] = np.einsum("pco,pci->oi", R(gz), R(acts[l]))
        gb[l] = gz[:, 0].sum(0)
        g = np.einsum("pco,oi->pci", R(gz), R(params.W[l]))
    # g: gradient w.r.t. the encoded features [P, 5, levels * F]
    spec = params.spec
    gg = np.zeros_like(params.grid)
    for l, (slots, cw) in enumerate(enc_cache):
        ge = g[:, :, l * spec.features:(l + 1) * spec.features]     # [P, 5, F]
        contrib = np.einsum("pcq,pcf->pqf", cw, ge)                  # [P, 8, F]
        np.add.at(gg[l], slots.reshape(-1), contrib.reshape(-1, spec.features))
    return loss(out, target, wch), gg, gW, gb


def init_params(spec: SurrogateSpec, seed: int = 0, grid_scale: float = 1e-4):
    """Deterministic initial parameters (splitmix64 streams): grid U(-s, s),
    weights U(-1/sqrt(in), 1/sqrt(in)), biases 0."""
    from paper_1708_02645_gb300 import inputs
    grid = (2.0 * inputs.uniform01(seed, spec.levels * spec.table * spec.features) - 1.0)
    grid = grid.reshape(spec.levels, spec.table, spec.features) * grid_scale
    widths = spec.widths()
    W, b = [], []
    for l in range(len(widths) - 1):
        fan_in = widths[l]
        u = inputs.uniform01(seed + 1 + l, widths[l + 1] * fan_in).reshape(widths[l + 1], fan_in)
        W.append((2.0 * u - 1.0) / math.sqrt(fan_in))
        b.append(np.zeros(widths[l + 1]))
    return SurrogateParams(spec, grid, W, b)


def as_float32(params: SurrogateParams) -> SurrogateParams:
    """The parameters rounded to FP32 (what a device copy holds), in FP64."""
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return SurrogateParams(params.spec, f(params.grid), [f(w) for w in params.W], [f(b) for b in params.b])
