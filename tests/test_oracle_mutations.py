"""Plant plausible mistakes in a copy of the oracle and check the pins catch each one.

The oracle's own source is never modified: each mutant is a textual edit of a
temporary copy, compiled next to it and loaded in place of the real library for
the duration of one test.
"""
import os

import pytest

import pins

MUTANTS = {
    "imag sign flipped": ("Fl[2 * k + 1] += u * c - q * s;", "Fl[2 * k + 1] += u * c + q * s;"),
    "U sin term dropped": ("Fl[2 * k] += q * c + u * s;", "Fl[2 * k] += q * c;"),
    "unweighted lambda0": ("swl += w * lambda2[i];", "swl += lambda2[i];"),
    "weights not applied to data": ("double q = w * Ql[i], u = w * Ul[i];", "double q = Ql[i], u = Ul[i];"),
    "factor 2 missing in phase": ("double theta = 2.0 * phi[k] * d;\n                double c",
                                  "double theta = phi[k] * d;\n                double c"),
    "K not applied": ("Fl[2 * k] *= K; Fl[2 * k + 1] *= K;", ""),
    "lambda0 dropped in synth": ("double d = lambda2[i] - lambda0sq;\n            for (int32_t k = 0; k < nphi; ++k) {\n                double theta",
                                 "double d = lambda2[i];\n            for (int32_t k = 0; k < nphi; ++k) {\n                double theta"),
    "rmsf conjugated": ("R[2 * k + 1] -= w * sin(theta);", "R[2 * k + 1] += w * sin(theta);"),
    "peak ties to last": ("if (best < 0 || m > bestm)", "if (best < 0 || m >= bestm)"),
    "LOS stride wrong": ("const double *Ql = Q + (size_t)l * (size_t)nchan;", "const double *Ql = Q + (size_t)l;"),
    "flagged channels not skipped": ("if (w == 0.0) continue;               /* flagged", "/* flagged"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(oracle_mod, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "rms_oracle.c")).read()
    assert src.count(old) >= 1, "mutation anchor not found: " + name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new, 1))
    so = oracle_mod.compile_variant(str(mut), str(tmp_path / "libmutant.so"))
    caught = []
    with oracle_mod.use_library(so):
        for pname, check in pins.PINS.items():
            try:
                check(oracle_mod)
            except AssertionError:
                caught.append(pname)
    assert caught, "planted mistake '%s' passed every pin" % name
