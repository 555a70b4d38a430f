"""Planted mistakes in the oracle must fail at least one pin.

Each case copies the oracle's C source, changes one expression into a
plausible mistake (a dropped term, a wrong sign, a wrong index, a transposed
operand), compiles the copy on the CPU, and runs the pins of
``tests/pins.py`` against it.  This shows the pins would catch that mistake
in the real oracle.  Nothing here touches a GPU.
"""
import functools
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "blip_oracle.c")

MUTANTS = [
    ("gradient uses J instead of J^T",
     "jb->J[0 + c] * dg[0] + jb->J[3 + c] * dg[1] + jb->J[6 + c] * dg[2]",
     "jb->J[3 * c + 0] * dg[0] + jb->J[3 * c + 1] * dg[1] + jb->J[3 * c + 2] * dg[2]"),
    ("Laplacian drops the xy cross term",
     "hg[0][1] = hg[1][0] = b1[0][kx] * b1[1][ky] * b0[2][kz];",
     "hg[0][1] = hg[1][0] = 0.0;"),
    ("Laplacian metric J J instead of J J^T",
     "s += J[3 * a + c] * J[3 * b + c];",
     "s += J[3 * a + c] * J[3 * c + b];"),
    ("outer-piece derivative sign flipped",
     "(x > 0 ? -0.5 : 0.5) * d * d",
     "(x > 0 ? 0.5 : -0.5) * d * d"),
    ("B(0) constant wrong",
     "return 2.0 / 3.0 - ax * ax + 0.5 * ax * ax * ax;",
     "return 0.65 - ax * ax + 0.5 * ax * ax * ax;"),
    ("second derivative outer piece wrong",
     "if (ax <= 2.0) return 2.0 - ax;",
     "if (ax <= 2.0) return 2.0 - 2.0 * ax;"),
    ("stencil starts one site late",
     "int sx = (base[0] - 1 + kx + n1) % n1;",
     "int sx = (base[0] + kx + n1) % n1;"),
    ("y index wrapped with n1",
     "int sy = (base[1] - 1 + ky + n2) % n2;",
     "int sy = (base[1] - 1 + ky + n1) % n1;"),
    ("table axes transposed",
     "(((size_t)sx * n2 + sy) * n3 + sz)",
     "(((size_t)sz * n2 + sy) * n1 + sx)"),
    ("stencil distances mirrored",
     "double x = t[a] + 1.0 - (double)k;",
     "double x = t[a] - 2.0 + (double)k;"),
    ("fractional coordinate uses A^T",
     "double u = jb->Ainv[3 * a + 0] * r[0] + jb->Ainv[3 * a + 1] * r[1]\n"
     "                 + jb->Ainv[3 * a + 2] * r[2];",
     "double u = jb->Ainv[0 + a] * r[0] + jb->Ainv[3 + a] * r[1]\n"
     "                 + jb->Ainv[6 + a] * r[2];"),
    ("grid scale n missing from J",
     "J[3 * a + c] = (double)grid[a] * Ainv[3 * a + c];",
     "J[3 * a + c] = (double)grid[c] * Ainv[3 * a + c];"),
    # the rounding scale C_o = sum_s |W_o(s)| |a_ls| (absmag): an inflated
    # scale would silently loosen every GPU parity bound built on it
    ("absmag: gradient weights made absolute before the Jacobian contraction",
     "double w = W[k], aw = fabs(W[k]);",
     "double w = W[k], aw = (k >= 1 && k <= 3)\n"
     "                        ? jb->norm * (fabs(jb->J[k - 1] * dg[0]) + fabs(jb->J[2 + k] * dg[1])\n"
     "                                      + fabs(jb->J[5 + k] * dg[2]))\n"
     "                        : fabs(W[k]);"),
    ("absmag: Laplacian weight made absolute term by term",
     "double w = W[k], aw = fabs(W[k]);",
     "double aw = fabs(W[k]);\n"
     "                    if (k == 4) {\n"
     "                        aw = 0.0;\n"
     "                        for (int a = 0; a < 3; ++a)\n"
     "                            for (int b = 0; b < 3; ++b) aw += fabs(jb->M[3 * a + b] * hg[a][b]);\n"
     "                        aw *= jb->norm;\n"
     "                    }\n"
     "                    double w = W[k];"),
    ("absmag: factor 2 on the derivative kinds",
     "double w = W[k], aw = fabs(W[k]);",
     "double w = W[k], aw = (k ? 2.0 : 1.0) * fabs(W[k]);"),
    ("absmag: signed coefficients",
     "am[l] += aw * fabs(c[l]);",
     "am[l] += aw * c[l];"),
]

TOL = {
    "check_bspline_closed_forms": 1e-15, "check_bspline_continuity": 1e-8,
    "check_bspline_derivatives_fd": 1e-9, "check_partition_of_unity": 1e-13,
    "check_polynomial_reproduction": 1e-12, "check_plane_wave_nodes": 1e-12,
    "check_finite_differences": 1e-7, "check_vs_bruteforce": 1e-13,
    "check_translation": 1e-12, "check_absmag_vs_bruteforce": 1e-12,
    "check_absmag_closed_forms": 1e-13,
}


def _failing_pins(lib):
    ev = functools.partial(oracle.eval_stencil, _lib=lib)
    failed = []
    for name, tol in TOL.items():
        f = getattr(pins, name)
        try:
            err = f(lib) if "bspline" in name else f(ev)
        except Exception:          # a crash also counts as caught
            failed.append(name)
            continue
        if not (err < tol):
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_every_pin():
    assert _failing_pins(oracle.lib()) == []


@pytest.mark.parametrize("label,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, label, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not found: {label}"
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c99",
                           "-D_POSIX_C_SOURCE=200809L", "-o", str(so), str(c), "-lm"])
    failed = _failing_pins(oracle.load(str(so)))
    assert failed, f"no pin caught: {label}"


def test_bruteforce_mutant_is_caught(monkeypatch):
    """A wrong B-spline in Oracle B breaks its agreement with Oracle A."""
    good = oracle.brute.bspline
    monkeypatch.setattr(oracle.brute, "bspline", lambda x: good(x * 1.01))
    assert pins.check_vs_bruteforce() > 1e-6
