"""FP64 CPU oracle of the THC-oo-K orbital gradient (the vo block of K).

TEST INFRASTRUCTURE (see ``oracle/thc_oracle.py`` for who may import it).

THC-oo-K fits the interpolation vectors to the occupied pair products
(Eq. orbprodoo), so the kernel V^q depends on the occupied orbitals, and the
orbital gradient of the exchange energy has, beside the term the build
already forms, the terms that come from that dependence (Sec. 2.3, the
``K_ai`` expression; Algorithm 2's ``dM/dtheta`` step).  This module states
that gradient by its definition: the derivative of the THC-oo-K exchange
energy with respect to an occupied-virtual rotation of the orbitals, with
the interpolation points fixed and the fit and the kernel redone.

* ``energy``: E_x(C) in plain numpy, the kernel refitted from the orbitals on
  the grid (``setup_oracle.fit_kernel``) and the build of ``thc_oracle``.
* ``vo_gradient``: g^k[a, i] = dE/dRe(theta^k[a, i]) + i dE/dIm(theta^k[a, i])
  for ``C^k -> C^k + Cv^k theta^k`` (the first order of a unitary rotation
  between occupied and virtual orbitals), from the same pipeline restated
  in torch (CPU, FP64) and differentiated by its autograd, with or without
  the kernel's dependence on the orbitals.
* ``explicit_gradient``: the closed form of the term with the kernel held
  fixed, ``g = -(4 / N_k) Cv^H (K C)`` with ``K C`` the build's output (the
  first term of the ``K_ai`` expression, scaled for this gradient).

A problem is a dict with ``lattice`` (3 x 3), ``grid`` (3), ``mesh`` (3),
``kfrac`` (N_k x 3), ``Xg`` (N_k, N, N_g) the Bloch basis on the whole grid
and ``points`` (N_P) grid indices of the interpolation points.
"""
from __future__ import annotations

import numpy as np

from . import setup_oracle as S
from . import thc_oracle as O


def grid_orbitals(prob: dict, C: np.ndarray) -> np.ndarray:
    """U[(k, i), r] = u^k_i(r) = exp(-i k.r) sum_mu Xg^k[mu, r] C^k[mu, i]."""
    lat = np.asarray(prob["lattice"], dtype=float)
    r = S.grid_frac(prob["grid"]) @ lat
    kc = np.asarray(prob["kfrac"]) @ S.recip_vectors(lat)
    psi = np.einsum("kmr,kmi->kir", prob["Xg"], C)
    ph = np.exp(-1j * (kc @ r.T))                   # (N_k, N_g)
    return (psi * ph[:, None, :]).reshape(-1, r.shape[0])


def energy(prob: dict, C: np.ndarray, V: np.ndarray | None = None) -> float:
    """THC-oo-K E_x of the orbitals C: the kernel refitted from them at the
    problem's points (or V, when given), then the build (Algorithm 2)."""
    if V is None:
        V = S.fit_kernel(prob["lattice"], prob["grid"], prob["mesh"], grid_orbitals(prob, C), prob["points"])
    Xp = np.ascontiguousarray(prob["Xg"][:, :, prob["points"]])
    return float(O.build(Xp, C, V, prob["mesh"], route="direct")["Ex"])


def explicit_gradient(prob: dict, C: np.ndarray, Cv: np.ndarray, V: np.ndarray) -> np.ndarray:
    """-(4 / N_k) Cv^{kH} (K C)^k for the kernel V held fixed.

    With E = -(1/N_k) sum_{k,k'} sum_PQ conj(D^k) D^k' V^{k'-k} (a real form,
    as V^{-q} = conj(V^q)), dE = -(4/N_k) Re sum conj(Y^k) dPsi^k with
    Y = M Psi, and dPsi^k = X^{kT} Cv^k theta^k; so dE/dRe(theta) + i
    dE/dIm(theta) = -(4/N_k) Cv^H conj(X) Y = -(4/N_k) Cv^H (K C)."""
    Xp = np.ascontiguousarray(prob["Xg"][:, :, prob["points"]])
    KC = O.build(Xp, C, V, prob["mesh"], route="direct")["KC"]
    nk = C.shape[0]
    return -(4.0 / nk) * np.einsum("kma,kmi->kai", Cv.conj(), KC)


# ----------------------------------------------------------------------------
# the same pipeline in torch (CPU, FP64), differentiated by autograd
# ----------------------------------------------------------------------------

def _kernel_torch(prob: dict, xi, torch):
    """setup_oracle.kernel_from_xi restated on torch tensors: V[q, P, Q] of
    the interpolation vectors xi[P, r] (Sec. 2.2), the symmetric G set and the
    mean over the minimum-image representatives of a zone-boundary q."""
    lat = np.asarray(prob["lattice"], dtype=float)
    grid, mesh, points = tuple(prob["grid"]), tuple(prob["mesh"]), np.asarray(prob["points"])
    B = S.recip_vectors(lat)
    vol = abs(np.linalg.det(lat))
    ng, nk, npts = int(np.prod(grid)), int(np.prod(mesh)), len(points)
    rP = (S.grid_frac(grid) @ lat)[points]
    gm = S.symmetric_gset(grid)
    flat = torch.from_numpy(np.ravel_multi_index(tuple((gm % np.array(grid)).T), grid))
    xh = torch.fft.fftn(xi.to(torch.complex128).reshape((npts,) + grid), dim=(1, 2, 3))
    xh = xh.reshape(npts, ng)[:, flat] * (vol / ng)
    Vs = []
    for qco in O.mesh_coords(mesh):
        reps = S.representatives(qco, mesh)
        acc = 0
        for qr in reps:
            qc = qr @ B
            v = torch.from_numpy(np.sqrt(S.coulomb((gm + qr[None, :]) @ B))).to(torch.complex128)
            ph = torch.from_numpy(np.exp(-1j * (rP @ qc)))
            A = xh * v[None, :] * ph[:, None]
            acc = acc + (A @ A.conj().T) / len(reps)
        Vs.append(acc / (nk * vol))
    return torch.stack(Vs)


def _energy_torch(prob: dict, C, V_fixed, torch):
    """E_x of the orbitals C (a torch tensor): the kernel refitted from C at
    the problem's points (isdf_fit, kernel_from_xi) unless V_fixed is given,
    then the five steps of the build."""
    mesh, points = tuple(prob["mesh"]), torch.from_numpy(np.asarray(prob["points"]))
    Xg = torch.from_numpy(prob["Xg"])
    nk = C.shape[0]
    if V_fixed is None:
        lat = np.asarray(prob["lattice"], dtype=float)
        r = S.grid_frac(prob["grid"]) @ lat
        kc = np.asarray(prob["kfrac"]) @ S.recip_vectors(lat)
        ph = torch.from_numpy(np.exp(-1j * (kc @ r.T)))
        U = (torch.einsum("kmr,kmi->kir", Xg, C) * ph[:, None, :]).reshape(-1, r.shape[0])
        ArP = (U.conj().T @ U[:, points]).abs() ** 2              # A(r, r_P)
        Sm = ArP[points]                                          # the ISDF metric A(r_P, r_Q)
        xi = torch.linalg.solve(Sm, ArP.T)                        # xi[P, r] (real, symmetric S)
        V = _kernel_torch(prob, xi, torch)
    else:
        V = torch.from_numpy(V_fixed)
    Psi = torch.einsum("kmp,kmi->kpi", Xg[:, :, points], C)
    D = Psi @ Psi.conj().transpose(1, 2)
    qi = np.array([[O.q_index(mesh, k, kp) for kp in range(nk)] for k in range(nk)])
    M = torch.stack([sum(D[kp] * V[int(qi[k, kp])] for kp in range(nk)) for k in range(nk)])
    Y = M @ Psi
    return -(Psi.conj() * Y).sum().real / nk


def vo_gradient(prob: dict, C: np.ndarray, Cv: np.ndarray, V_fixed: np.ndarray | None = None) -> np.ndarray:
    """g^k[a, i] = dE/dRe(theta^k[a, i]) + i dE/dIm(theta^k[a, i]) at theta = 0
    for C^k -> C^k + Cv^k theta^k, by autograd of the torch restatement; the
    kernel refitted with the orbitals (the THC-oo-K orbital gradient, Sec. 2.3)
    unless V_fixed is given (then only the explicit term)."""
    import torch
    nk, _, n = C.shape
    nv = Cv.shape[2]
    tx = torch.zeros((nk, nv, n), dtype=torch.float64, requires_grad=True)
    ty = torch.zeros((nk, nv, n), dtype=torch.float64, requires_grad=True)
    theta = torch.complex(tx, ty)
    Ct = torch.from_numpy(C) + torch.from_numpy(Cv) @ theta
    E = _energy_torch(prob, Ct, V_fixed, torch)
    gx, gy = torch.autograd.grad(E, (tx, ty))
    return (gx + 1j * gy).numpy()
