"""Comparison helpers for GPU-vs-oracle parity.

Tolerances (FP32 accumulation, stated per output group):
* kernel parity (oracle run on the coefficients exactly as stored):
  max|d| / max|ref| <= 1e-5 per group (V, G, H or L), and per element
  |d| <= 64 * 2^-24 * beta + 2^-24 * |ref|, where beta = sum |W| |c| over
  the window (the FP32 evaluation of a 64-term sum of products errs by a
  small multiple of 2^-24 beta);
* storage-format error (oracle run on the original FP64 coefficients):
  per element |d| <= u_fmt * beta + 64 * 2^-24 * beta (+ 2^-25 * sum|W| for
  FP16, whose subnormals have an absolute spacing of 2^-24), with
  u_bf16 = 2^-8 and u_f16 = 2^-11 (unit roundoff of each format).
"""
import numpy as np

U32 = 2.0 ** -24
UNIT_ROUNDOFF = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
MAX_REL = 1e-5

GROUPS = {
    0: {"V": [0]},
    1: {"V": [0], "G": [1, 2, 3], "L": [4]},
    2: {"V": [0], "G": [1, 2, 3], "H": [4, 5, 6, 7, 8, 9]},
}


def as_rows(a, kind):
    """[P, N] -> [P, 1, N] so that every kind has a component axis."""
    a = np.asarray(a)
    return a[:, None, :] if kind == 0 else a


def errors(got, ref, kind):
    """max-rel and RMS-rel error per group (max|d|/max|ref|, ||d||/||ref||)."""
    got, ref = as_rows(got, kind).astype(np.float64), as_rows(ref, kind)
    res = {}
    for name, comps in GROUPS[kind].items():
        d = got[:, comps] - ref[:, comps]
        r = ref[:, comps]
        mx = max(np.abs(r).max(), 1e-300) if r.size else 1.0
        nr = max(np.sqrt((r ** 2).sum()), 1e-300) if r.size else 1.0
        res[name] = {"max_rel": float(np.abs(d).max() / mx) if d.size else 0.0,
                     "rms_rel": float(np.sqrt((d ** 2).sum()) / nr) if d.size else 0.0}
    return res


def assert_kernel_parity(got, ref, beta, kind, what=""):
    got = as_rows(got, kind).astype(np.float64)
    ref = as_rows(ref, kind)
    beta = as_rows(beta, kind)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.isfinite(got).all(), f"{what}: non-finite output"
    err = errors(got, ref, kind)
    for name, e in err.items():
        assert e["max_rel"] <= MAX_REL, f"{what}: group {name} max-rel {e['max_rel']:.3g} > {MAX_REL}"
    bound = 64 * U32 * beta + U32 * np.abs(ref)
    d = np.abs(got - ref)
    bad = d > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: element {tuple(i)} |d|={d[tuple(i)]:.3g} > bound "
                             f"{bound[tuple(i)]:.3g} ({bad.sum()} elements)")
    return err


def assert_format_error(got, ref64, beta, wsum, kind, fmt, what=""):
    got = as_rows(got, kind).astype(np.float64)
    ref64 = as_rows(ref64, kind)
    beta = as_rows(beta, kind)
    wsum = as_rows(wsum, kind)
    bound = UNIT_ROUNDOFF[fmt] * beta + 64 * U32 * beta
    if fmt == "f16":
        bound = bound + 2.0 ** -25 * wsum
    d = np.abs(got - ref64)
    bad = d > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: element {tuple(i)} |d|={d[tuple(i)]:.3g} > bound "
                             f"{bound[tuple(i)]:.3g} ({bad.sum()} elements)")
    return errors(got, ref64, kind)


def round_to_bf16_bits(x):
    """FP64 -> BF16 bit patterns, one round-to-nearest-even step (normal range)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                          # x = m 2^e, |m| in [0.5, 1)
    r = np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)  # 8 significant bits, ties to even
    return (r.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def bf16_bits_to_f64(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def stored_values(coefs64, fmt):
    """The coefficient values a table of format fmt holds (as FP64), and the
    array to upload so that the library stores exactly those values."""
    if fmt == "f32":
        up = np.asarray(coefs64, dtype=np.float32)
        return up.astype(np.float64), up, None
    if fmt == "f16":
        up = np.asarray(coefs64, dtype=np.float64).astype(np.float16)
        return up.astype(np.float64), up, None
    bits = round_to_bf16_bits(coefs64)
    return bf16_bits_to_f64(bits), bits, "bf16"
