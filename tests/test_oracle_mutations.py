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


# ---------------------------------------------------------------------------
# mutants of the setup oracle's Coulomb kernel and q representatives: both
# sides of the full-grid identity share these, so they are caught by the
# closed-form pins instead
# ---------------------------------------------------------------------------

from oracle import setup_oracle as S  # noqa: E402


def _coulomb_2pi(K):
    K2 = np.einsum("gi,gi->g", K, K)
    out = np.zeros_like(K2)
    nz = K2 > 1e-12
    out[nz] = 2.0 * np.pi / K2[nz]
    return out


def _coulomb_first_power(K):
    K2 = np.einsum("gi,gi->g", K, K)
    out = np.zeros_like(K2)
    nz = K2 > 1e-12
    out[nz] = 4.0 * np.pi / np.sqrt(K2[nz])
    return out


def _representatives_unwrapped(qco, mesh):
    return [np.array([(int(qco[a]) % mesh[a]) / mesh[a] for a in range(3)])]


SETUP_MUTANTS = {
    "coulomb_2pi": ("coulomb", _coulomb_2pi),
    "coulomb_1_over_K": ("coulomb", _coulomb_first_power),
    "q_not_minimum_image": ("representatives", _representatives_unwrapped),
}


def _coulomb_pins_fail() -> list:
    fails = []
    if pins.check_gaussian_self_energy(8.0)["rel"] > 1e-12:
        fails.append("gaussian")
    lattice = np.diag([6.95, 8.9, 6.45])
    for mesh in [(2, 2, 2), (3, 3, 3)]:
        if pins.check_plane_wave_kernel(lattice, (8, 8, 8), mesh, (1, 0, 0)) > 1e-13:
            fails.append(f"plane_wave{mesh}")
    return fails


@pytest.mark.parametrize("name", sorted(SETUP_MUTANTS))
def test_setup_mutant_is_caught(monkeypatch, name):
    fn, mutant = SETUP_MUTANTS[name]
    monkeypatch.setattr(S, fn, mutant)
    assert _coulomb_pins_fail(), f"mutant {name} passed every Coulomb pin"


def test_setup_unmutated_passes():
    assert not _coulomb_pins_fail()
