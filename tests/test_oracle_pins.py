"""Pins of the FP64 oracle to facts other than the oracle itself.

The paper (arXiv 1708.02645) evaluates the orbitals phi_i(r) of the Slater
matrix and their gradients and Laplacians (Sec. 3, Alg. 1 "ratio" and
"derivatives") with a 3-D cubic B-spline (cited in Sec. 3, not printed).
It prints no worked example and no output values, so the oracle is pinned by
the mathematics of the uniform cubic B-spline:

* partition of unity: constant coefficients give a constant value and zero
  derivatives;
* impulse response: a single unit coefficient gives B3 products with the
  textbook values 2/3, 1/6, 23/48 and the derivative values -1/2, -2, 1;
* polynomial reproduction (Marsden's identity for B3 centred on integers):
  coefficients 1, m, m^2 - 1/3, m^3 - m reproduce 1, u, u^2, u^3, so a tensor
  product of cubics is reproduced exactly with all derivatives;
* plane waves at grid nodes: the symbol of B3 at integers is (2 + cos th)/3;
* C2 continuity across cell faces; finite differences of V and G;
* periodic wrap; linearity and orbital independence;
* a brute-force global sum over all periodic images with the piecewise B3,
  written independently of the oracle's windowed weights.

Each check is a function of an evaluator, so that test_oracle_mutants.py can
run the same checks on deliberately broken copies of the oracle.
"""
import math

import numpy as np
import pytest

from paper_1708_02645_gb300 import inputs

V, GX, GY, GZ, HXX, HXY, HXZ, HYY, HYZ, HZZ = range(10)
KIND_V, KIND_VGL, KIND_VGH = 0, 1, 2
# derivative orders (x, y, z) of each VGH component
ORDERS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0),
          (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]


def oracle_ev(coefs, pos, kind=KIND_VGH, lib=None):
    import oracle
    return oracle.spo_eval(coefs, pos, kind, lib=lib)


# ---------------------------------------------------------------------------
# independent brute force: global sum with the piecewise B3 and its
# derivatives, folded over all periodic images
# ---------------------------------------------------------------------------
def b3(s, order):
    a = np.abs(s)
    if order == 0:
        return np.where(a < 1, 2.0 / 3.0 - a * a + 0.5 * a ** 3,
                        np.where(a < 2, (2.0 - a) ** 3 / 6.0, 0.0))
    if order == 1:
        return np.where(a < 1, -2.0 * s + 1.5 * s * a,
                        np.where(a < 2, -np.sign(s) * (2.0 - a) ** 2 / 2.0, 0.0))
    return np.where(a < 1, -2.0 + 3.0 * a, np.where(a < 2, 2.0 - a, 0.0))


def brute_force_vgh(coefs, pos):
    """phi(r) = sum over m in Z^3 of c[m mod n] prod_d B3(r_d n_d - m_d),
    with d/dr_d = n_d d/du_d.  Every image m within n+3 cells of u is summed."""
    coefs = np.asarray(coefs, dtype=np.float64)
    nx, ny, nz, N = coefs.shape
    ns = (nx, ny, nz)
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pos.shape[0], 10, N))
    for p, r in enumerate(pos):
        fold = []
        for d in range(3):
            n = ns[d]
            u = r[d] * n
            m = np.arange(math.floor(u) - n - 3, math.floor(u) + n + 4)
            f = np.zeros((3, n))
            for k in range(3):
                np.add.at(f[k], np.mod(m, n), b3(u - m, k) * float(n) ** k)
            fold.append(f)
        for q, (kx, ky, kz) in enumerate(ORDERS):
            out[p, q] = np.einsum("i,j,k,ijkn->n", fold[0][kx], fold[1][ky], fold[2][kz], coefs)
    return out


def _scale(ref):
    return np.maximum(np.abs(ref).max(axis=(0, 2), keepdims=True), 1e-300)


def assert_close_groups(got, ref, rtol, what=""):
    """max |got - ref| per component <= rtol * max |ref| of that component"""
    err = np.abs(got - ref).max(axis=(0, 2))
    sc = np.abs(ref).max(axis=(0, 2))
    bad = [(q, err[q], sc[q]) for q in range(ref.shape[1]) if err[q] > rtol * max(sc[q], 1.0)]
    assert not bad, f"{what}: components off (index, max err, scale): {bad}"


# ---------------------------------------------------------------------------
# checks (each takes an evaluator ev(coefs, pos, kind))
# ---------------------------------------------------------------------------
def check_partition_of_unity(ev):
    grid = (5, 6, 7)
    consts = np.array([2.5, -1.25, 0.0, 7.0])
    c = np.broadcast_to(consts, grid + (4,)).copy()
    pos = np.concatenate([inputs.uniform_positions(64, 11), inputs.wide_positions(64, 12)])
    out = ev(c, pos, KIND_VGH)
    assert np.abs(out[:, V] - consts).max() < 1e-13
    assert np.abs(out[:, 1:]).max() < 1e-11  # derivatives of a constant vanish


def check_impulse_response(ev):
    nx, ny, nz = 8, 16, 32   # node coordinates m/n are exact in binary
    m0 = (3, 5, 7)
    c = np.zeros((nx, ny, nz, 1))
    c[m0 + (0,)] = 1.0
    node = np.array([m0[0] / nx, m0[1] / ny, m0[2] / nz])
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    pts = np.array([node,
                    node + [h[0], 0, 0],          # neighbour along x
                    node + [0, -h[1], 0],         # neighbour along -y
                    node + [h[0], h[1], 0],       # diagonal neighbour
                    node + [0.5 * h[0], 0, 0],    # half-way along x
                    node + [2 * h[0], 0, 0]])     # outside the support
    out = ev(c, pts, KIND_VGH)[:, :, 0]
    b0, b1, bh = 2.0 / 3.0, 1.0 / 6.0, 23.0 / 48.0   # B3(0), B3(1), B3(1/2)
    d1, dh = -0.5, -0.625                            # B3'(1), B3'(1/2)
    e = {
        (0, V): b0 ** 3, (0, GX): 0.0, (0, GY): 0.0, (0, GZ): 0.0,
        (0, HXX): -2.0 * nx * nx * b0 * b0, (0, HYY): -2.0 * ny * ny * b0 * b0,
        (0, HZZ): -2.0 * nz * nz * b0 * b0, (0, HXY): 0.0,
        (1, V): b1 * b0 * b0, (1, GX): d1 * nx * b0 * b0, (1, HXX): 1.0 * nx * nx * b0 * b0,
        (2, V): b1 * b0 * b0, (2, GY): -d1 * ny * b0 * b0, (2, GX): 0.0,
        (3, V): b1 * b1 * b0, (3, HXY): d1 * nx * d1 * ny * b0,
        (4, V): bh * b0 * b0, (4, GX): dh * nx * b0 * b0,
        (5, V): 0.0, (5, GX): 0.0, (5, HXX): 0.0,
    }
    for (i, q), val in e.items():
        assert abs(out[i, q] - val) < 1e-12 * max(1.0, abs(val)), (i, q, out[i, q], val)


def _marsden(m, alpha):
    """coefficient of the polynomial sum_k alpha_k u^k in the B3 basis"""
    mu = [np.ones_like(m), m, m * m - 1.0 / 3.0, m ** 3 - m]
    return sum(alpha[k] * mu[k] for k in range(4))


def check_polynomial_reproduction(ev):
    ns = (9, 10, 11)
    N = 4
    rng = np.random.default_rng(5)
    alpha = rng.uniform(-1, 1, size=(N, 3, 4))  # orbital, axis, degree
    axes = [np.arange(n, dtype=np.float64) for n in ns]
    c = np.ones(ns + (N,))
    for j in range(N):
        fx = _marsden(axes[0], alpha[j, 0])
        fy = _marsden(axes[1], alpha[j, 1])
        fz = _marsden(axes[2], alpha[j, 2])
        c[..., j] = fx[:, None, None] * fy[None, :, None] * fz[None, None, :]
    # cells whose window does not wrap: i in [1, n-3]
    P = 200
    u = np.stack([rng.integers(1, n - 2, size=P) + rng.uniform(0, 1, size=P) for n in ns], axis=1)
    pos = u / np.array(ns)
    out = ev(c, pos, KIND_VGH)
    for j in range(N):
        vals = []
        for d in range(3):
            a = alpha[j, d]
            x = u[:, d]
            p0 = a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3
            p1 = (a[1] + 2 * a[2] * x + 3 * a[3] * x ** 2) * ns[d]
            p2 = (2 * a[2] + 6 * a[3] * x) * ns[d] ** 2
            vals.append((p0, p1, p2))
        for q, (kx, ky, kz) in enumerate(ORDERS):
            exp = vals[0][kx] * vals[1][ky] * vals[2][kz]
            err = np.abs(out[:, q, j] - exp).max()
            assert err < 1e-10 * max(1.0, np.abs(exp).max()), (j, q, err)


def check_plane_wave_nodes(ev):
    ns = np.array([8, 12, 10])
    k = np.array([1, 2, -3])
    th = 2 * np.pi * k / ns
    mg = np.stack(np.meshgrid(*[np.arange(n) for n in ns], indexing="ij"), -1)
    phase = np.exp(1j * (mg @ th))
    c = np.stack([phase.real, phase.imag], -1)  # two orbitals: cos and sin
    nodes = np.array([[1, 2, 3], [0, 0, 0], [7, 11, 9], [4, 6, 5]])
    out = ev(c, nodes / ns, KIND_VGH)
    sym = (2 + np.cos(th)) / 3.0
    d1 = 1j * np.sin(th) * ns
    d2 = (2 * np.cos(th) - 2) * ns * ns
    for i, m in enumerate(nodes):
        e = np.exp(1j * (m @ th))
        f = [[sym[d], d1[d], d2[d]] for d in range(3)]
        for q, (kx, ky, kz) in enumerate(ORDERS):
            z = e * f[0][kx] * f[1][ky] * f[2][kz]
            scale = max(1.0, float(np.max(ns)) ** (kx + ky + kz))
            assert abs(out[i, q, 0] - z.real) < 1e-12 * scale, (i, q)
            assert abs(out[i, q, 1] - z.imag) < 1e-12 * scale, (i, q)


def check_generator_plane_waves(ev):
    """The plane-wave input recipe evaluated at nodes gives the closed form
    Re sum_j a_j e^{2 pi i k_j m/n} prod_d (2 + cos(2 pi k_jd / n_d))/3."""
    ns = (8, 8, 16)
    N = 3
    c = inputs.plane_wave_coefs(*ns, N, seed=77)
    k, a = inputs.plane_wave_spec(N, seed=77)
    nodes = np.array([[1, 2, 3], [7, 0, 15], [4, 4, 8]])
    out = ev(c, nodes / np.array(ns), KIND_V)
    for i, m in enumerate(nodes):
        for j in range(N):
            th = 2 * np.pi * k[j] / np.array(ns)
            z = np.sum(a[j] * np.exp(1j * (th @ m)) * np.prod((2 + np.cos(th)) / 3.0, axis=1))
            assert abs(out[i, j] - z.real) < 1e-12


def check_c2_continuity(ev):
    ns = np.array([6, 7, 9])
    c = inputs.uniform_coefs(*ns, 3, seed=3)
    rng = np.random.default_rng(8)
    eps = 1e-11
    for d in range(3):
        base = rng.uniform(0, 1, size=(20, 3))
        base[:, d] = rng.integers(0, ns[d], size=20) / ns[d]   # on a cell face
        lo, hi = base.copy(), base.copy()
        lo[:, d] -= eps
        hi[:, d] += eps
        a, b = ev(c, lo, KIND_VGH), ev(c, hi, KIND_VGH)
        # first derivatives of H are bounded by ~ n^3 |c|, so the jump over
        # 2 eps is tiny unless the window shift is wrong
        tol = 1e-6 * float(ns.max()) ** 2
        assert np.abs(a - b).max() < tol, (d, np.abs(a - b).max())


def check_finite_differences(ev):
    ns = np.array([6, 8, 7])
    c = inputs.uniform_coefs(*ns, 2, seed=4)
    rng = np.random.default_rng(9)
    r = rng.uniform(-0.5, 1.5, size=(40, 3))
    delta = 1e-6
    base = ev(c, r, KIND_VGH)
    gscale = np.abs(base[:, GX:GZ + 1]).max()
    hscale = np.abs(base[:, HXX:]).max()
    hidx = {(0, 0): HXX, (0, 1): HXY, (0, 2): HXZ, (1, 1): HYY, (1, 2): HYZ, (2, 2): HZZ}
    for d in range(3):
        e = np.zeros(3)
        e[d] = delta
        up, dn = ev(c, r + e, KIND_VGH), ev(c, r - e, KIND_VGH)
        fd = (up - dn) / (2 * delta)
        assert np.abs(fd[:, V] - base[:, GX + d]).max() < 1e-5 * gscale, d
        for d2 in range(3):
            q = hidx[tuple(sorted((d, d2)))]
            # O(delta) where the stencil straddles a knot (third derivative jumps)
            assert np.abs(fd[:, GX + d2] - base[:, q]).max() < 1e-4 * hscale, (d, d2)


def check_periodic_wrap(ev):
    ns = (5, 7, 6)
    c = inputs.uniform_coefs(*ns, 3, seed=5)
    r = inputs.uniform_positions(50, seed=6).astype(np.float64)
    base = ev(c, r, KIND_VGH)
    for shift in ([1, 0, 0], [0, -1, 0], [0, 0, 3], [-2, 2, -1]):
        out = ev(c, r + np.array(shift, dtype=np.float64), KIND_VGH)
        assert np.array_equal(out, base), shift


def check_brute_force(ev):
    for ns, N, seed in (((4, 4, 4), 2, 21), ((5, 4, 7), 3, 22), ((7, 5, 4), 2, 23)):
        c = inputs.uniform_coefs(*ns, N, seed=seed)
        pos = np.concatenate([inputs.uniform_positions(24, seed + 100),
                              inputs.wide_positions(24, seed + 200)])
        ref = brute_force_vgh(c, pos)
        got = ev(c, pos, KIND_VGH)
        assert_close_groups(got, ref, 1e-13, f"brute force {ns}")


def check_linearity_and_orbitals(ev):
    ns = (6, 5, 7)
    A = inputs.uniform_coefs(*ns, 4, seed=31)
    B = inputs.uniform_coefs(*ns, 4, seed=32)
    r = inputs.wide_positions(40, seed=33)
    al, be = 0.75, -1.5
    lhs = ev(al * A + be * B, r, KIND_VGH)
    rhs = al * ev(A, r, KIND_VGH) + be * ev(B, r, KIND_VGH)
    assert_close_groups(lhs, rhs, 1e-13, "linearity")
    perm = np.array([2, 0, 3, 1])
    assert np.array_equal(ev(A[..., perm], r, KIND_VGH), ev(A, r, KIND_VGH)[..., perm])


def check_kinds_agree(ev):
    ns = (6, 6, 5)
    c = inputs.uniform_coefs(*ns, 5, seed=41)
    r = inputs.wide_positions(30, seed=42)
    h = ev(c, r, KIND_VGH)
    g = ev(c, r, KIND_VGL)
    v = ev(c, r, KIND_V)
    assert np.array_equal(v, h[:, V])
    assert np.array_equal(g[:, :4], h[:, :4])
    assert np.array_equal(g[:, 4], h[:, HXX] + h[:, HYY] + h[:, HZZ])


ALL_CHECKS = [check_partition_of_unity, check_impulse_response, check_polynomial_reproduction,
              check_plane_wave_nodes, check_generator_plane_waves, check_c2_continuity,
              check_finite_differences, check_periodic_wrap, check_brute_force,
              check_linearity_and_orbitals, check_kinds_agree]


@pytest.mark.parametrize("check", ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(oracle_lib, check):
    check(oracle_ev)


# ---------------------------------------------------------------------------
# condition sums beta_q = sum over the window of |W_q| |c| (the scale of the
# rounding error of any evaluation of the same sums; they set the per-element
# bounds of every GPU parity test).  Each check takes an oracle-like module
# `o` (spo_eval, condition, spo_ratio, spo_ratio_condition), so that the
# mutant tests can run them on broken copies.
#
# Closed forms, derived from the cubic B-spline pieces on one cell (t in
# [0, 1], derivatives with respect to u = r n):
#   sum_a |w_a|   = 1                        (w_a >= 0, partition of unity)
#   sum_a |w'_a|  = 1 + 2 t (1 - t)          (w'_0, w'_1 <= 0 <= w'_2, w'_3 and
#                                             sum w' = 0: twice the positive part,
#                                             w'_2 + w'_3 = (1 + 2t - 2t^2)/2)
#   sum_a |w''_a| = max(2, 4 - 6 t, 6 t - 2) (w''_0 = 1-t, w''_3 = t >= 0;
#                                             w''_1 = 3t-2, w''_2 = 1-3t change
#                                             sign at t = 2/3 and 1/3)
# With |c| = kappa_j for every node, beta of a tensor-product weight is
# kappa_j times the product of these one-axis sums (times n_d per derivative).
# ---------------------------------------------------------------------------
def _frac(pos, ns):
    """t_d = u_d - floor(u_d), u_d = r_d n_d (exact for FP32 positions)"""
    u = np.asarray(pos, dtype=np.float64).reshape(-1, 3) * np.asarray(ns, dtype=np.float64)
    return u - np.floor(u)


def _abs_sum_d1(t):
    return 1.0 + 2.0 * t * (1.0 - t)


def _abs_sum_d2(t):
    return np.maximum(2.0, np.maximum(4.0 - 6.0 * t, 6.0 * t - 2.0))


def brute_force_condition(coefs, pos):
    """beta_q(r) = sum over m in Z^3 of |prod_d n_d^k_d B3^(k_d)(u_d - m_d)|
    |c[m mod n]| for the ten VGH derivative orders, with the piecewise B3 and
    every integer m within 3 cells of u (no window bookkeeping)."""
    coefs = np.abs(np.asarray(coefs, dtype=np.float64))
    ns = coefs.shape[:3]
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pos.shape[0], 10, coefs.shape[3]))
    for p, r in enumerate(pos):
        ms, bs = [], []
        for d in range(3):
            u = r[d] * ns[d]
            m = np.arange(math.floor(u) - 3, math.floor(u) + 4)
            ms.append(np.mod(m, ns[d]))
            bs.append([b3(u - m, k) * float(ns[d]) ** k for k in range(3)])
        cw = coefs[np.ix_(ms[0], ms[1], ms[2])]          # |c| of every image in range
        for q, (kx, ky, kz) in enumerate(ORDERS):
            w = np.abs(np.einsum("i,j,k->ijk", bs[0][kx], bs[1][ky], bs[2][kz]))
            out[p, q] = np.einsum("ijk,ijkn->n", w, cw)
    return out


def _signed_constant_table(ns, kappa, seed):
    """|c| = kappa_j at every node, random signs"""
    rng = np.random.default_rng(seed)
    sign = rng.choice([-1.0, 1.0], size=tuple(ns) + (len(kappa),))
    return sign * np.asarray(kappa, dtype=np.float64)


def _condition_positions(ns, seed):
    nodes = np.stack([np.arange(6) % n / n for n in ns], axis=1)   # t = 0 on every axis
    thirds = np.array([[1 / 3, 2 / 3, 0.5]]) / np.asarray(ns)      # kinks of sum |w''|
    return np.concatenate([inputs.uniform_positions(40, seed).astype(np.float64),
                           inputs.wide_positions(40, seed + 1).astype(np.float64),
                           nodes, thirds])


def check_condition_closed_forms(o):
    ns = np.array([5, 6, 7])
    kappa = np.array([0.5, 1.5, 2.0])
    c = _signed_constant_table(ns, kappa, 61)
    pos = _condition_positions(ns, 62)
    t = _frac(pos, ns)
    s1 = _abs_sum_d1(t) * ns                 # [P, 3]: n_d sum |w'|
    s2 = _abs_sum_d2(t) * ns * ns            # n_d^2 sum |w''|
    one = np.ones_like(t)
    per_axis = [one, s1, s2]
    want = np.empty((pos.shape[0], 10, 3))
    for q, (kx, ky, kz) in enumerate(ORDERS):
        f = per_axis[kx][:, 0] * per_axis[ky][:, 1] * per_axis[kz][:, 2]
        want[:, q] = f[:, None] * kappa
    got = o.condition(c, pos, KIND_VGH)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), np.abs(got - want).max()
    lap = (s2.sum(axis=1))[:, None] * kappa
    g = o.condition(c, pos, KIND_VGL)
    assert np.abs(g[:, :4] - want[:, :4]).max() <= 1e-13 * np.abs(want[:, :4]).max()
    assert np.abs(g[:, 4] - lap).max() <= 1e-13 * np.abs(lap).max()
    assert np.abs(o.condition(c, pos, KIND_V) - kappa).max() <= 1e-14
    # at a node every first-derivative sum is n_d (1/2 + 0 + 1/2)
    at_nodes = o.condition(c, pos[80:86], KIND_VGH)
    for d in range(3):
        assert np.abs(at_nodes[:, GX + d] - ns[d] * kappa).max() <= 1e-13 * ns[d]


def check_condition_of_nonnegative_table_is_value(o):
    """c >= 0: every |W_V c| = W_V c, so beta_V equals V itself."""
    ns = (6, 5, 7)
    c = inputs.uniform_coefs(*ns, 4, seed=63) + 1.0          # in [0, 2)
    pos = _condition_positions(ns, 64)
    v = o.spo_eval(c, pos, KIND_V)
    b = o.condition(c, pos, KIND_V)
    assert np.abs(b - v).max() <= 1e-14 * np.abs(v).max()
    # and beta dominates |output| for any signs (triangle inequality)
    c2 = inputs.uniform_coefs(*ns, 4, seed=65)
    h = o.spo_eval(c2, pos, KIND_VGH)
    bh = o.condition(c2, pos, KIND_VGH)
    assert (np.abs(h) <= bh * (1 + 1e-13) + 1e-300).all()


def check_condition_brute_force(o):
    for ns, N, seed in (((4, 4, 4), 2, 66), ((5, 4, 7), 3, 67), ((7, 5, 4), 2, 68)):
        c = inputs.uniform_coefs(*ns, N, seed=seed)
        pos = _condition_positions(ns, seed + 100)
        ref = brute_force_condition(c, pos)
        got = o.condition(c, pos, KIND_VGH)
        assert_close_groups(got, ref, 1e-13, f"condition brute force {ns}")


def check_ratio_condition(o):
    """beta of a ratio: sum_j |row_j| beta_V,j.  For rows >= 0 and c >= 0 it
    is the ratio itself; for |c| = kappa_j it is sum_j |row_j| kappa_j."""
    ns, N, R = (6, 7, 5), 4, 3
    rng = np.random.default_rng(69)
    pos = _condition_positions(ns, 70)
    P = pos.shape[0]
    row_of = rng.integers(0, R, size=P)
    rows = rng.uniform(0.1, 1.0, size=(R, N))
    c = inputs.uniform_coefs(*ns, N, seed=71) + 1.0
    rho = o.spo_ratio(c, pos, rows, row_of=row_of)
    beta = o.spo_ratio_condition(c, pos, rows, row_of=row_of)
    assert np.abs(beta - rho).max() <= 1e-13 * np.abs(rho).max()
    kappa = np.array([0.25, 1.0, 3.0, 0.5])
    cs = _signed_constant_table(ns, kappa, 72)
    srows = rows * rng.choice([-1.0, 1.0], size=rows.shape)
    beta = o.spo_ratio_condition(cs, pos, srows, row_of=row_of)
    want = np.abs(srows[row_of]) @ kappa
    assert np.abs(beta - want).max() <= 1e-13 * want.max()
    # row_of = None means row p for position p
    beta = o.spo_ratio_condition(cs, pos[:R], srows)
    assert np.abs(beta - np.abs(srows) @ kappa).max() <= 1e-13 * want.max()


CONDITION_CHECKS = [check_condition_closed_forms, check_condition_of_nonnegative_table_is_value,
                    check_condition_brute_force, check_ratio_condition]


@pytest.mark.parametrize("check", CONDITION_CHECKS, ids=lambda f: f.__name__)
def test_condition_pin(oracle_lib, check):
    check(oracle_lib)


def test_brute_force_condition_reproduces_closed_values(oracle_lib):
    """The brute force itself: at a node with c = 1 everywhere, beta_V = 1,
    beta_Gx = n (B3'(+-1) = -+1/2), beta_Hxx = 4 n^2 (|B3''| = 1, 2, 1)."""
    c = np.ones((4, 5, 6, 1))
    out = brute_force_condition(c, np.array([[0.25, 0.4, 0.5]]))
    assert abs(out[0, V, 0] - 1.0) < 1e-15
    assert abs(out[0, GX, 0] - 4.0) < 1e-14
    assert abs(out[0, HXX, 0] - 4.0 * 16.0) < 1e-12
    assert abs(out[0, HYZ, 0] - 5.0 * 6.0) < 1e-12


def test_brute_force_is_independent_of_window(oracle_lib):
    """The brute force itself reproduces B3's closed values (impulse at node)."""
    c = np.zeros((4, 4, 4, 1))
    c[1, 1, 1, 0] = 1.0
    out = brute_force_vgh(c, np.array([[0.25, 0.25, 0.25], [0.5, 0.25, 0.25]]))
    assert abs(out[0, V, 0] - 8.0 / 27.0) < 1e-15
    assert abs(out[1, V, 0] - (1.0 / 6.0) * (4.0 / 9.0)) < 1e-15
    assert abs(out[1, GX, 0] - (-0.5 * 4) * (4.0 / 9.0)) < 1e-14


def test_oracle_rejects_bad_arguments(oracle_lib):
    import oracle
    with pytest.raises(ValueError):
        oracle.spo_eval(np.zeros((3, 4, 4, 1)), np.zeros((1, 3)))


def test_oracle_empty_inputs(oracle_lib):
    import oracle
    out = oracle.spo_eval(np.zeros((4, 4, 4, 2)), np.zeros((0, 3)))
    assert out.shape == (0, 10, 2)
    out = oracle.spo_eval(np.zeros((4, 4, 4, 0)), np.zeros((3, 3)))
    assert out.shape == (3, 10, 0)


def test_ratio_is_the_determinant_ratio(oracle_lib):
    """eq. md_lemma: with A(i, j) = phi_i(r_j), moving electron k to r' gives
    det(A') / det(A) = (row k of A^-1) . phi(r').  Checked against
    numpy.linalg.det on the spline's own orbital matrix."""
    import oracle
    ns, N = (7, 6, 8), 9
    c = inputs.uniform_coefs(*ns, N, seed=51)
    r = inputs.uniform_positions(N, seed=52).astype(np.float64)      # N electrons
    A = oracle.spo_eval(c, r, KIND_V).T                               # A[i, j] = phi_i(r_j)
    Ainv = np.linalg.inv(A)
    moves = inputs.wide_positions(N, seed=53).astype(np.float64)     # r'_k for each k
    rho = oracle.spo_ratio(c, moves, Ainv, row_of=np.arange(N))       # row k for move k
    phi_new = oracle.spo_eval(c, moves, KIND_V)                       # [k, i]
    for k in range(N):
        A2 = A.copy()
        A2[:, k] = phi_new[k]
        exact = np.linalg.det(A2) / np.linalg.det(A)
        assert abs(rho[k] - exact) < 1e-9 * max(1.0, abs(exact)), (k, rho[k], exact)


def test_ratio_reduces_to_values_for_unit_rows(oracle_lib):
    import oracle
    c = inputs.uniform_coefs(5, 5, 6, 4, seed=54)
    pos = inputs.wide_positions(12, seed=55).astype(np.float64)
    v = oracle.spo_eval(c, pos, KIND_V)
    eye = np.eye(4)
    for j in range(4):
        rho = oracle.spo_ratio(c, pos, eye[j:j + 1], row_of=np.zeros(12, dtype=int))
        assert np.array_equal(rho, v[:, j])


def test_prefilter_interpolates_at_the_nodes(oracle_lib):
    """The spline of the prefiltered coefficients passes through the samples
    at every grid node (V), independently checked by the oracle's window
    sums; on tiny grids the prefilter also equals the dense solve of the
    per-axis cyclic systems (c[m-1] + 4 c[m] + c[m+1]) / 6 = f[m]."""
    import oracle
    ns, N = (5, 6, 7), 3
    f = inputs.uniform_coefs(*ns, N, seed=71)
    c = oracle.prefilter(f)
    nodes = np.stack(np.meshgrid(*[np.arange(n) / n for n in ns], indexing="ij"), -1).reshape(-1, 3)
    v = oracle.spo_eval(c, nodes, KIND_V)
    assert np.abs(v - f.reshape(-1, N)).max() < 1e-12
    # dense per-axis solve
    d = np.array(f)
    for ax, n in enumerate(ns):
        A = np.zeros((n, n))
        for j in range(n):
            A[j, (j - 1) % n] += 1 / 6
            A[j, j] += 4 / 6
            A[j, (j + 1) % n] += 1 / 6
        d = np.moveaxis(np.linalg.solve(A, np.moveaxis(d, ax, 0).reshape(n, -1)).reshape(
            np.moveaxis(d, ax, 0).shape), 0, ax)
    assert np.abs(d - c).max() < 1e-12


def test_prefilter_plane_wave_symbol(oracle_lib):
    """Samples cos(th . m) are divided by prod_d (2 + cos th_d) / 3."""
    import oracle
    ns = (8, 6, 10)
    k = np.array([1, 2, 3])
    th = 2 * np.pi * k / np.array(ns)
    m = np.stack(np.meshgrid(*[np.arange(n) for n in ns], indexing="ij"), -1)
    f = np.cos((m * th).sum(-1))[..., None]
    c = oracle.prefilter(f)
    want = f / np.prod((2 + np.cos(th)) / 3)
    assert np.abs(c - want).max() < 1e-12
