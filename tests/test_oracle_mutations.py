"""Plant plausible mistakes in the oracle (on the CPU) and check that at least
one pin catches each.  This shows the pins can fail, so their passing means
something.  Every mutant is applied with monkeypatch and undone after."""
import numpy as np
import pytest

from oracle import thc_oracle as O

import pins


def _conv_wrong_sign(D, V, mesh):
    """q = k - k' instead of k' - k."""
    nk = D.shape[0]
    M = np.zeros_like(D)
    for k in range(nk):
        for kp in range(nk):
            M[k] += D[kp] * V[O.q_index(mesh, kp, k)]
    return M


def _density_no_conj(Psi):
    return np.stack([Psi[k] @ Psi[k].T for k in range(Psi.shape[0])])


def _backproject_no_conj(X, Y):
    return np.stack([X[k] @ Y[k] for k in range(X.shape[0])])


def _energy_no_norm(Psi, Y):
    return -np.sum(Psi.conj() * Y)


def _conv_dropped_term(D, V, mesh):
    """Leaves out the k' = k term (q = 0)."""
    nk = D.shape[0]
    M = np.zeros_like(D)
    for k in range(nk):
        for kp in range(nk):
            if kp != k:
                M[k] += D[kp] * V[O.q_index(mesh, k, kp)]
    return M


def _collocate_conj(X, C):
    return np.stack([X[k].T.conj() @ C[k] for k in range(X.shape[0])])


MUTANTS = {
    "q_sign": ("kconv_direct", _conv_wrong_sign),
    "density_conj": ("density", _density_no_conj),
    "backproject_conj": ("backproject", _backproject_no_conj),
    "energy_norm": ("exchange_energy", _energy_no_norm),
    "dropped_q0": ("kconv_direct", _conv_dropped_term),
    "collocate_conj": ("collocate", _collocate_conj),
}


def _any_pin_fails() -> list:
    fails = []
    for mesh, grid in [((3, 3, 3), (8, 8, 8)), ((3, 2, 4), (8, 8, 8))]:
        r = pins.check_full_grid(mesh, grid)
        if r["ex_rel"] > 1e-8 or r["kc_rel"] > 1e-8:
            fails.append(f"full_grid{mesh}")
    return fails


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(monkeypatch, name):
    fn, mutant = MUTANTS[name]
    monkeypatch.setattr(O, fn, mutant)
    assert _any_pin_fails(), f"mutant {name} passed every pin"


def test_unmutated_passes():
    assert not _any_pin_fails()
