"""Planted mistakes in the oracle must fail at least one pin.

Each mutant is a copy of oracle/spo_oracle.c with one plausible slip (a wrong
constant, a dropped term, a wrong sign or index, a transposed operand),
compiled on the CPU into a temporary library and run through the same
checks as the real oracle.  Every mutant keeps all memory accesses in bounds.
"""
import os
import subprocess

import numpy as np
import pytest

import test_oracle_pins as pins

MUTANTS = {
    "weight_constant": ("- 6.0 * t * t + 4.0) / 6.0", "- 6.0 * t * t + 3.0) / 6.0"),
    "dweight_sign": ("dw[2] = 0.5 * (-3.0 * t * t", "dw[2] = 0.5 * (3.0 * t * t"),
    "d2weight_scale": ("d2w[0] = s * nn * nn;", "d2w[0] = s * nn;"),
    "window_offset": ("long xa = (ix + a - 1 + nx) % nx;", "long xa = (ix + a + nx) % nx;"),
    "dropped_corner": ("for (int g = 0; g < 4; ++g) {\n                long zg",
                       "for (int g = 0; g < 3; ++g) {\n                long zg"),
    "transposed_hessian": ("W[5] = dwx[a] * dwy[b] * wz[g];", "W[5] = dwx[a] * wy[b] * dwz[g];"),
    "swapped_axes_index": ("(((size_t)xa * ny + yb) * nz + zg) * (size_t)N;\n                double W[10];",
                           "(((size_t)yb * nx + xa) * nz + zg) * (size_t)N;\n                double W[10];"),
    "gradient_axis": ("W[2] = wx[a] * dwy[b] * wz[g];", "W[2] = dwx[a] * wy[b] * wz[g];"),
    "laplacian_term": ("h[4 * N + j] + h[7 * N + j] + h[9 * N + j]",
                       "h[4 * N + j] + h[7 * N + j] + h[8 * N + j]"),
    "value_path_index": ("double W = wx[a] * wy[b] * wz[g];", "double W = wx[a] * wy[b] * wz[b];"),
    "fraction_sign": ("double t = u - fl;", "double t = fl - u + 1.0;"),
    "ny_for_nz": ("basis_weights(tz, nz, wz, dwz, d2wz);\n\n    for (long k",
                  "basis_weights(tz, ny, wz, dwz, d2wz);\n\n    for (long k"),
    # slips in the condition sums (oracle_spo_condition), which set every
    # per-element bound of the GPU parity tests
    "cond_dropped_abs_c": ("hq[j] += aw * fabs(c[j]);", "hq[j] += aw * c[j];"),
    "cond_dropped_abs_w": ("double aw = fabs(W[q]);", "double aw = W[q];"),
    "cond_weights_only": ("hq[j] += aw * fabs(c[j]);", "hq[j] += aw;"),
    "cond_wrong_component": ("                    W[6] = dwx[a] * wy[b] * dwz[g];",
                             "                    W[6] = dwx[a] * dwy[b] * wz[g];"),
    "cond_stray_factor_n": ("double aw = fabs(W[q]);", "double aw = fabs(W[q]) * nx;"),
    "cond_window_offset": ("            long xa = (ix + a - 1 + nx) % nx;",
                           "            long xa = (ix + a + nx) % nx;"),
}

# slips in the Python side of the oracle (oracle/__init__.py)
PY_MUTANTS = {
    "laplacian_beta_rows": ("(b[:, 4] + b[:, 7] + b[:, 9])", "(b[:, 4] + b[:, 5] + b[:, 9])"),
    "laplacian_beta_whole_hessian": ("(b[:, 4] + b[:, 7] + b[:, 9])", "b[:, 4:10].sum(axis=1)"),
    "ratio_condition_signed_rows": ("rows = np.abs(np.asarray(rows, dtype=np.float64))",
                                    "rows = np.asarray(rows, dtype=np.float64)"),
    "ratio_condition_ignores_row_of": (
        "rows = np.abs(np.asarray(rows, dtype=np.float64))\n"
        "    idx = np.arange(b.shape[0]) if row_of is None else np.asarray(row_of)",
        "rows = np.abs(np.asarray(rows, dtype=np.float64))\n    idx = np.arange(b.shape[0])"),
}


def oracle_variant(py_source, lib):
    """A copy of the oracle package's module, executed from `py_source` and
    bound to the compiled library `lib`."""
    import types

    import oracle
    mod = types.ModuleType("oracle_variant")
    mod.__file__ = oracle.__file__
    exec(compile(py_source, oracle.__file__, "exec"), mod.__dict__)
    mod._lib = lib
    return mod


def failed_pins(o):
    """names of the pins (evaluator and condition checks) the module o fails"""
    def ev(coefs, pos, kind=pins.KIND_VGH):
        return o.spo_eval(coefs, pos, kind)

    caught = []
    for check, arg in [(c, ev) for c in pins.ALL_CHECKS] + [(c, o) for c in pins.CONDITION_CHECKS]:
        try:
            with np.errstate(all="ignore"):
                check(arg)
        except (AssertionError, IndexError, ValueError):   # wrong values, or unusable output
            caught.append(check.__name__)
    return caught


@pytest.fixture(scope="module")
def oracle_source():
    import oracle
    with open(os.path.join(os.path.dirname(oracle.__file__), "spo_oracle.c")) as f:
        return f.read()


@pytest.fixture(scope="module")
def oracle_py_source():
    import oracle
    with open(oracle.__file__) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, oracle_source, oracle_py_source, tmp_path, oracle_lib):
    old, new = MUTANTS[name]
    assert oracle_source.count(old) >= 1, f"mutation site for {name} not found"
    src = oracle_source.replace(old, new, 1)
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(so), str(cpath), "-lm"], check=True)
    o = oracle_variant(oracle_py_source, oracle_lib.load_variant(str(so)))
    assert failed_pins(o), f"mutant {name} passed every pin"


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_python_mutant_is_caught(name, oracle_py_source, oracle_lib):
    old, new = PY_MUTANTS[name]
    assert oracle_py_source.count(old) == 1, f"mutation site for {name} not found or ambiguous"
    o = oracle_variant(oracle_py_source.replace(old, new), oracle_lib._load())
    assert failed_pins(o), f"mutant {name} passed every pin"


def test_unmutated_copies_pass(oracle_source, oracle_py_source, oracle_lib):
    """the mutation machinery itself: an unchanged copy passes every pin"""
    assert failed_pins(oracle_variant(oracle_py_source, oracle_lib._load())) == []
