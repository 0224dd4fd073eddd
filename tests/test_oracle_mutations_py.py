"""Plant plausible mistakes in copies of the Python oracle modules and check that
the pins catch each one (the counterpart of test_oracle_mutations.py for the C
oracle).  The oracle's own files are never modified: each mutant is a textual
edit of the module source, executed as a separate module and passed to, or
patched into, the pin tests for the duration of one test.
"""
import inspect
import types

import pytest

import test_clean_oracle
import test_net_oracle
import test_oracle_pins

MUTANTS = {
    # oracle/__init__.py: sub-grid peak and chi0
    "refine: vertex sign": ("oracle", "ts = min(max(-c1 / (2.0 * c2)", "ts = min(max(c1 / (2.0 * c2)"),
    "refine: parabola on |F|^2": ("oracle", "y = np.abs(F[l].astype(np.complex128))",
                                   "y = np.abs(F[l].astype(np.complex128)) ** 2"),
    "refine: offset from the left sample": ("oracle", "t = phi[k - 1:k + 2] - phi[k]\n",
                                            "t = phi[k - 1:k + 2] - phi[k - 1]\n"),
    "refine: height not re-evaluated": ("oracle", "abs_ref[l] = np.polyval([c2, c1, c0], ts)", "abs_ref[l] = c0"),
    "chi0: lambda_0 term sign": ("oracle", "- np.asarray(phi_peak, dtype=np.float64) * lambda0sq",
                                 "+ np.asarray(phi_peak, dtype=np.float64) * lambda0sq"),
    "chi0: half angle dropped": ("oracle", "x = 0.5 * np.arctan2(F_peak.imag, F_peak.real)",
                                 "x = np.arctan2(F_peak.imag, F_peak.real)"),
    # oracle/clean.py: RM-CLEAN
    "clean: gain not applied": ("clean", "cr, ci = g * rr[j], g * ri[j]", "cr, ci = rr[j], ri[j]"),
    "clean: RMSF conjugated": ("clean", "ri = np.subtract(ri, np.add(np.multiply(cr, si), np.multiply(ci, sr)))",
                               "ri = np.subtract(ri, np.subtract(np.multiply(ci, sr), np.multiply(cr, si)))"),
    "clean: threshold on |res|^2 against threshold": ("clean", "if not m2[j] >= thr2:", "if not m2[j] >= thr:"),
    "clean: beam width": ("clean", "beam = np.exp(-4.0 * math.log(2.0)", "beam = np.exp(-math.log(2.0)"),
    "clean: component at the wrong bin": ("clean", "comp[l, j] += complex(cr, ci)", "comp[l, j - 1] += complex(cr, ci)"),
    # oracle/net.py: the network and the learned peak map
    "net: ReLU mask dropped in backward": ("net", "da1 = dh * (a1 > 0)", "da1 = dh"),
    "net: batch mean missing in dz": ("net", "    dz /= n\n", "\n"),
    "net: Q and U swapped": ("net", "x[:, 0::2] = q\n    x[:, 1::2] = u", "x[:, 0::2] = u\n    x[:, 1::2] = q"),
    "net: RMS over one channel too many": ("net", "axis=1) / len(act))", "axis=1) / (len(act) + 1))"),
    "net: window mass one bin short": ("net", "bi - halfwin):bi + halfwin + 1]", "bi - halfwin):bi + halfwin]"),
    "net: centre not clamped at the top": ("net", "2 * (nbins - 1) - width // 2 + 1", "2 * (nbins - 1)"),
    "net: edge fallback on the last point missed": ("net", "k <= 0 or k == width - 1", "k <= 0"),
}


def _mutant(module, old, new):
    src = inspect.getsource(module)
    assert src.count(old) >= 1, "mutation anchor not found"
    m = types.ModuleType(module.__name__ + "_mutant")
    m.__file__ = module.__file__
    exec(compile(src.replace(old, new, 1), module.__file__, "exec"), m.__dict__)
    return m


def _run(tests, *args):
    caught = []
    for t in tests:
        try:
            t(*args)
        except Exception as e:          # an assertion, or an error the mistake causes
            caught.append((t.__name__, type(e).__name__))
    return caught


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_python_oracle_mutant_is_caught(oracle_mod, monkeypatch, name):
    where, old, new = MUTANTS[name]
    if where == "oracle":
        mut = _mutant(oracle_mod, old, new)
        tests = [getattr(test_oracle_pins, n) for n in dir(test_oracle_pins)
                 if n.startswith("test_") and ("refine" in n or "chi0" in n)]
        caught = _run(tests, mut)
    elif where == "clean":
        from oracle import clean
        monkeypatch.setattr(test_clean_oracle, "oc", _mutant(clean, old, new))
        tests = [getattr(test_clean_oracle, n) for n in dir(test_clean_oracle) if n.startswith("test_")]
        caught = _run(tests, oracle_mod)
    else:
        from oracle import net
        monkeypatch.setattr(test_net_oracle, "net", _mutant(net, old, new))
        tests = [getattr(test_net_oracle, n) for n in dir(test_net_oracle) if n.startswith("test_")]
        caught = []
        for t in tests:
            args = (oracle_mod,) if "oracle_mod" in inspect.signature(t).parameters else ()
            caught += _run([t], *args)
    assert caught, "planted mistake '%s' passed every pin" % name


@pytest.mark.parametrize("where", ["oracle", "clean", "net"])
def test_unmutated_copies_pass_every_pin(oracle_mod, monkeypatch, where):
    # the harness itself: a copy with no edit must pass every pin it is checked against
    anchor = {"oracle": "def refine_peak(", "clean": "def clean(", "net": "def forward("}[where]
    if where == "oracle":
        mut = _mutant(oracle_mod, anchor, anchor)
        tests = [getattr(test_oracle_pins, n) for n in dir(test_oracle_pins)
                 if n.startswith("test_") and ("refine" in n or "chi0" in n)]
        assert len(tests) >= 7
        assert _run(tests, mut) == []
    elif where == "clean":
        from oracle import clean
        monkeypatch.setattr(test_clean_oracle, "oc", _mutant(clean, anchor, anchor))
        tests = [getattr(test_clean_oracle, n) for n in dir(test_clean_oracle) if n.startswith("test_")]
        assert len(tests) >= 4
        assert _run(tests, oracle_mod) == []
    else:
        from oracle import net
        monkeypatch.setattr(test_net_oracle, "net", _mutant(net, anchor, anchor))
        tests = [getattr(test_net_oracle, n) for n in dir(test_net_oracle) if n.startswith("test_")]
        assert len(tests) >= 7
        for t in tests:
            args = (oracle_mod,) if "oracle_mod" in inspect.signature(t).parameters else ()
            assert _run([t], *args) == [], t.__name__
