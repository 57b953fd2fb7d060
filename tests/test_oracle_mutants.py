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
}


@pytest.fixture(scope="module")
def oracle_source():
    import oracle
    with open(os.path.join(os.path.dirname(oracle.__file__), "spo_oracle.c")) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, oracle_source, tmp_path, oracle_lib):
    old, new = MUTANTS[name]
    assert oracle_source.count(old) >= 1, f"mutation site for {name} not found"
    src = oracle_source.replace(old, new, 1)
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(so), str(cpath), "-lm"], check=True)
    lib = oracle_lib.load_variant(str(so))

    def ev(coefs, pos, kind=pins.KIND_VGH):
        return pins.oracle_ev(coefs, pos, kind, lib=lib)

    caught = []
    for check in pins.ALL_CHECKS:
        try:
            with np.errstate(all="ignore"):
                check(ev)
        except AssertionError:
            caught.append(check.__name__)
    assert caught, f"mutant {name} passed every pin"
