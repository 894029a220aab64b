"""Plant plausible mistakes in the oracle (on the CPU, through monkeypatch)
and check that the closed-form pins catch each one."""
import numpy as np

from oracle import field, geometry, kress, operators, solvers
from tests import closed_forms as cf


def _disk_error(which, w=24.0, n=256):
    c = geometry.circle(n)
    R = kress.kress_weights(n)
    ms = np.arange(-int(w) - 10, int(w) + 11)
    S_ex, D_ex, _ = cf.disk_layer_eigenvalues(ms, w)
    row = operators.layer_rows(c, w, np.array([0]), which, R)[0]
    lam = np.array([np.sum(row * np.exp(1j * m * c.t)) for m in ms])
    return np.max(np.abs(lam - (S_ex if which == "S" else D_ex)))


def _point_source_error(bc, kind="kite", w=12.0, n=256):
    x0 = np.array([0.1, 0.05])
    c = geometry.make(kind, n)
    A = operators.cfie_matrix(c, w, w, bc)
    q = solvers.lu_solve(A, operators.point_source_rhs(c, w, x0, bc))
    pts = cf.ring(3.0, 16)
    return cf.rel(field.scattered_field(c, w, w, bc, q, pts), -cf.green(w, pts, x0))


def test_pins_pass_unpatched():
    assert _disk_error("S") < 1e-12
    assert _disk_error("D") < 1e-12
    assert _point_source_error("soft") < 1e-9
    assert _point_source_error("hard") < 1e-9


def test_dropped_euler_constant_is_caught(monkeypatch):
    monkeypatch.setattr(operators, "EULER_GAMMA", 0.0)
    assert _disk_error("S") > 1e-4


def test_flipped_curvature_term_is_caught(monkeypatch):
    orig = operators.layer_rows

    def flipped(curve, omega, rows, which, R=None):
        A = orig(curve, omega, rows, which, R)
        if which in ("D", "Dp"):
            rows = np.asarray(rows)
            A[np.arange(rows.size), rows] *= -1.0
        return A

    monkeypatch.setattr(operators, "layer_rows", flipped)
    assert _disk_error("D") > 1e-4


def test_swapped_double_layer_for_its_adjoint_is_caught(monkeypatch):
    """D and D' agree on the disk, so the pin must come from a non-circular curve."""
    orig = operators.layer_rows

    def swapped(curve, omega, rows, which, R=None):
        return orig(curve, omega, rows, "D" if which == "Dp" else which, R)

    monkeypatch.setattr(operators, "layer_rows", swapped)
    assert _point_source_error("hard") > 1e-4


def test_scaled_kress_weights_are_caught(monkeypatch):
    orig = kress.kress_weights
    monkeypatch.setattr(operators, "kress_weights", lambda n: 1.001 * orig(n))
    c = geometry.circle(64)
    R = operators.kress_weights(64)
    i = np.arange(64)
    s = np.sum(R[(0 - i) % 64] * np.exp(3j * c.t))
    assert abs(s - (-(2 * np.pi / 3))) > 1e-4
    assert _point_source_error("soft") > 1e-6


def test_wrong_hypersingular_sign_is_caught(monkeypatch):
    orig = operators.hypersingular_matrix
    monkeypatch.setattr(operators, "hypersingular_matrix", lambda c, w, S: -orig(c, w, S))
    assert _point_source_error("hard") > 1e-3
