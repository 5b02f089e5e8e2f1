"""The oracle's pins have teeth: each plausible slip planted in a copy of the oracle (a
dropped term, a flipped sign, a missing dt, theta or factor 2, a transposed operand, an
output one step late) makes at least one pin of that oracle module fail, while the
unchanged copy passes them all.  The slips are planted on the CPU, in a temporary copy;
the oracle itself is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the slip is, oracle file, text in it, the slipped text)
MUTATIONS = [
    ("theta dt R_D dropped from the electrode increment", "theta.py",
     "g -= (red.LD + dt * theta * red.RD) @ dD", "g -= red.LD @ dD"),
    ("coil source with the wrong sign", "theta.py",
     "g -= red.M0 @ (src[:, k + 1] - src[:, k])", "g += red.M0 @ (src[:, k + 1] - src[:, k])"),
    ("dt dropped from the resistive electrode term", "theta.py",
     "g -= dt * (red.RD @ iD[:, k])", "g -= red.RD @ iD[:, k]"),
    ("K^T M^D dropped from L_D", "theta.py",
     "LD = K.T @ L @ PE + K.T @ MD", "LD = K.T @ L @ PE"),
    ("modal c_n without theta", "theta.py",
     "1.0 / (tau + theta * dt)", "1.0 / (tau + dt)"),
    ("theta missing from Z", "theta.py",
     "Z = red.Li + dt * theta * red.Ri", "Z = red.Li + dt * red.Ri"),
    ("plain probe reads the electrode current one step early", "theta.py",
     "probes[:, k] = red.CK @ Ii + red.CPE @ iD[:, k + 1]",
     "probes[:, k] = red.CK @ Ii + red.CPE @ iD[:, k]"),
    ("transposed operand in the two-sided reduction", "theta.py",
     "A = sla.solve_triangular(CR, W.T, lower=True)", "A = sla.solve_triangular(CR, W, lower=True)"),
    ("modal a_n with theta in place of 1 - theta", "theta.py",
     "(tau - (1.0 - theta) * dt)", "(tau - theta * dt)"),
    ("adjoint: theta weights of the resistance gradient swapped", "adjoint.py",
     "gR -= dt * lam * (theta * I[:, k] + (1.0 - theta) * I[:, k - 1])",
     "gR -= dt * lam * ((1.0 - theta) * I[:, k] + theta * I[:, k - 1])"),
    ("adjoint: factor 2 of the misfit derivative dropped", "adjoint.py",
     "A @ lam_next + 2.0 * (C.T @ res[:, k - 1])", "A @ lam_next + (C.T @ res[:, k - 1])"),
    ("adjoint: source gradient with the wrong sign", "adjoint.py",
     "dsrc = mu[:, 1:] - mu[:, :-1]", "dsrc = mu[:, :-1] - mu[:, 1:]"),
    ("exact integrator: alternating series sign lost", "exponential.py",
     "term = -term * hs / (j + 1)", "term = term * hs / (j + 1)"),
    ("exact integrator: ramp term dropped", "exponential.py",
     "x = a * x + c0 * (U.T @ F0) + c1 * (U.T @ F1)", "x = a * x + c0 * (U.T @ F0)"),
    ("phasor: conjugate kernel", "phasor.py",
     "E = np.exp(-2j * np.pi", "E = np.exp(2j * np.pi"),
    ("phasor: factor 2 dropped", "phasor.py",
     "return (2.0 / T) * (E @ y.T)", "return (1.0 / T) * (E @ y.T)"),
]

PINS = {"theta.py": "test_oracle_pins.py", "adjoint.py": "test_oracle_adjoint.py",
        "exponential.py": "test_oracle_exponential.py", "phasor.py": "test_oracle_phasor.py"}


def _run_pins(tmp_path, module, old=None, new=None):
    work = tmp_path / "tree"
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle")
    shutil.copytree(os.path.join(ROOT, "workloads"), work / "workloads")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), work / "tests" / "golden")
    shutil.copy(os.path.join(ROOT, "tests", PINS[module]), work / "tests")
    (work / "tests" / "conftest.py").write_text(
        "import os, sys\n"
        "sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))\n")
    if old is not None:
        path = work / "oracle" / module
        text = path.read_text()
        assert text.count(old) == 1, old
        path.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        "tests/" + PINS[module]], cwd=work, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, r.stdout[-3000:]


@pytest.mark.parametrize("module", sorted(PINS))
def test_unchanged_copy_passes(tmp_path, module):
    code, out = _run_pins(tmp_path, module)
    assert code == 0, out


@pytest.mark.parametrize("what,module,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_slip_is_caught(tmp_path, what, module, old, new):
    code, out = _run_pins(tmp_path, module, old, new)
    assert code != 0, f"no pin caught: {what}\n{out}"
