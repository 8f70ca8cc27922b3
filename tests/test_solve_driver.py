"""The solve driver's checkpoint / resume wiring (host logic, no GPU): the engine and
the scheme are replaced by fakes that record what the driver passes them."""
import json
import sys

import numpy as np

from oracle import integrals as I
from paper_2012_15662_gb300 import solve
from paper_2012_15662_gb300.checkpoint import load_state
from synthetic import make_workload


class _FakeEngine:
    def __init__(self, w):
        self.nbf = w.system.nbf
        self.w = w
        self.closed = False

    def rhf(self, max_iter=200, tol=1e-8):
        return self.w.C.copy(), np.linspace(-1.0, 1.0, self.nbf), -11.0, 9, 1e-9

    def close(self):
        self.closed = True


def _run(monkeypatch, capsys, argv):
    w = make_workload("square4", I.overlap)
    eng = _FakeEngine(w)
    calls = []

    def fake_converge(e, C0, gamma0, diag0, exact=False, **kw):
        calls.append(dict(C0=np.array(C0), gamma0=np.array(gamma0), diag0=np.array(diag0), exact=exact))
        k = len(calls)
        return dict(C=np.array(C0) * (1.0 + 1e-3 * k), gamma=np.array(gamma0) + 0.01 * k, diag=np.array(diag0) - k,
                    E=-11.3 - 0.01 * k, outer=3 + k, converged=True, inner_total=10, seconds=0.1,
                    ms_per_inner=1.0, history=[])

    monkeypatch.setattr(solve.bd, "engine_and_workload", lambda name, prec: (eng, w))
    monkeypatch.setattr(solve, "converge", fake_converge)
    monkeypatch.setattr(sys, "argv", ["solve"] + argv)
    solve.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    return w, calls, line


def test_checkpoint_then_exact_restart_from_the_file(monkeypatch, capsys, tmp_path):
    ck = str(tmp_path / "ri")
    w, calls, line = _run(monkeypatch, capsys, ["--workload", "square4", "--forms", "fp64", "--checkpoint", ck])
    assert len(calls) == 1 and not calls[0]["exact"] and "rhf" in line
    st = load_state(ck, workload="square4", nbf=w.system.nbf)
    np.testing.assert_array_equal(st["C"], calls[0]["C0"] * 1.001)
    np.testing.assert_array_equal(st["gamma"], calls[0]["gamma0"] + 0.01)
    assert st["E"] == -11.31 and st["outer"] == 4 and st["form"] == "fp64"
    # resume: no RI run, the exact restart starts from the file and writes its own state
    ck2 = str(tmp_path / "again")
    _, calls2, line2 = _run(monkeypatch, capsys, ["--workload", "square4", "--forms", "", "--restart",
                                                  "--resume", ck, "--checkpoint", ck2])
    assert len(calls2) == 1 and calls2[0]["exact"]
    np.testing.assert_array_equal(calls2[0]["C0"], st["C"])
    np.testing.assert_array_equal(calls2[0]["gamma0"], st["gamma"])
    np.testing.assert_array_equal(calls2[0]["diag0"], st["diag"])
    assert line2["start"]["resumed_from"] == ck and line2["restart_exact"]["ri_error"] == st["E"] - (-11.31)
    ex = load_state(ck2 + "_exact", workload="square4")
    assert ex["form"] == "fp64-exact"
