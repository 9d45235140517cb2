"""FP64 CPU oracle of the learned interpolation-point proposal.

TEST INFRASTRUCTURE (see ``oracle/thc_oracle.py`` for who may import it).

The paper selects interpolation points by a deterministic decomposition
(Sec. 2.1) or by k-means on the density (Sec. 4); it has no learned part.
The network here is a small scorer of grid points: it proposes about
4 N_ISDF candidates, and the pivoted Cholesky of the occupied pair Gram
matrix (``setup_oracle.pivoted_cholesky``) then picks the points among them.
Everything below is a plain definition in float64:

* features of a grid point r: log(rho(r) + eps), log(|grad rho(r)| + eps) and
  the periodic minimum-image distance to the nearest atomic centre, with
  rho(r) = (1/N_k) sum_{k,i} |u^k_i(r)|^2 and the gradient by second-order
  central differences on the periodic grid;
* the network 3 -> 64 -> 64 -> 64 -> 1 with SiLU activations on standardised
  features, its output a logit;
* the loss: binary cross-entropy with logits, positives (grid points the
  full-grid pivoted Cholesky picks) weighted by pos_weight, averaged over the
  batch;
* analytic gradients by backpropagation, and one Adam step.

The parameter vector is laid out W1 [64][3], b1 [64], W2 [64][64], b2 [64],
W3 [64][64], b3 [64], W4 [64], b4 (8,641 values).
"""
from __future__ import annotations

import itertools

import numpy as np

H = 64
NPARAM = 3 * H + H + H * H + H + H * H + H + H + 1
EPS_FEAT = 1e-8


def split(params: np.ndarray):
    """Views W1, b1, W2, b2, W3, b3, W4, b4 of the flat parameter vector."""
    o = 0
    out = []
    for shape in ((H, 3), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)):
        n = int(np.prod(shape))
        out.append(params[o:o + n].reshape(shape))
        o += n
    assert o == NPARAM
    return out


def init_params(seed: int) -> np.ndarray:
    """Seeded initial weights: uniform in +-1/sqrt(fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    p = np.zeros(NPARAM)
    W1, b1, W2, b2, W3, b3, W4, b4 = split(p)
    W1[:] = rng.uniform(-1, 1, W1.shape) / np.sqrt(3)
    W2[:] = rng.uniform(-1, 1, W2.shape) / np.sqrt(H)
    W3[:] = rng.uniform(-1, 1, W3.shape) / np.sqrt(H)
    W4[:] = rng.uniform(-1, 1, W4.shape) / np.sqrt(H)
    return p


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------

def density(U: np.ndarray, nk: int) -> np.ndarray:
    """rho(r) = (1/N_k) sum_f |U[f, r]|^2 over the occupied f = (k, i)."""
    return np.sum(np.abs(U) ** 2, axis=0) / nk


def grad_norm(rho: np.ndarray, grid, lattice) -> np.ndarray:
    """|grad rho| from periodic second-order central differences along the
    three grid axes, taken to Cartesian with the reciprocal vectors
    (d f_a / d r = b_a / 2 pi)."""
    r3 = rho.reshape(grid)
    B = 2.0 * np.pi * np.linalg.inv(lattice).T
    g = np.zeros(r3.shape + (3,))
    for a in range(3):
        dfa = (np.roll(r3, -1, axis=a) - np.roll(r3, 1, axis=a)) * grid[a] / 2.0
        g += dfa[..., None] * (B[a] / (2.0 * np.pi))[None, None, None, :]
    return np.sqrt(np.sum(g ** 2, axis=-1)).ravel()


def nearest_centre(grid, lattice, centres: np.ndarray) -> np.ndarray:
    """Minimum-image distance from every grid point to the nearest centre."""
    axes = [np.arange(g) / g for g in grid]
    frac = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    cf = centres @ np.linalg.inv(lattice)
    best = np.full(frac.shape[0], np.inf)
    for c in cf:
        d = frac - c[None, :]
        d -= np.round(d)
        for n in itertools.product((-1, 0, 1), repeat=3):
            v = (d + np.array(n)[None, :]) @ lattice
            best = np.minimum(best, np.sqrt(np.sum(v ** 2, axis=1)))
    return best


def features(U: np.ndarray, nk: int, grid, lattice, centres) -> np.ndarray:
    """[N_g, 3]: log(rho + eps), log(|grad rho| + eps), nearest-centre distance."""
    rho = density(U, nk)
    return np.stack([np.log(rho + EPS_FEAT), np.log(grad_norm(rho, grid, lattice) + EPS_FEAT),
                     nearest_centre(grid, lattice, centres)], axis=1)


# ----------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------

def sigmoid(a):
    return 0.5 * (1.0 + np.tanh(0.5 * a))


def silu(a):
    return a * sigmoid(a)


def silu_grad(a):
    s = sigmoid(a)
    return s * (1.0 + a * (1.0 - s))


def softplus(a):
    return np.logaddexp(0.0, a)


def standardise(feat: np.ndarray, norm: np.ndarray) -> np.ndarray:
    """norm = (mean[3], std[3])."""
    return (feat - norm[:3][None, :]) / norm[3:][None, :]


def forward(params: np.ndarray, x: np.ndarray):
    """Logits z[n] of standardised features x[n, 3], and the layer values."""
    W1, b1, W2, b2, W3, b3, W4, b4 = split(params)
    a1 = x @ W1.T + b1
    h1 = silu(a1)
    a2 = h1 @ W2.T + b2
    h2 = silu(a2)
    a3 = h2 @ W3.T + b3
    h3 = silu(a3)
    z = h3 @ W4 + b4[0]
    return z, (x, a1, h1, a2, h2, a3, h3)


def loss(params, x, y, pos_weight: float) -> float:
    """Mean weighted BCE with logits: pos_weight y softplus(-z) + (1 - y) softplus(z)."""
    z, _ = forward(params, x)
    return float(np.mean(pos_weight * y * softplus(-z) + (1.0 - y) * softplus(z)))


def loss_grad(params, x, y, pos_weight: float):
    """(loss, d loss / d params) by backpropagation."""
    W1, b1, W2, b2, W3, b3, W4, b4 = split(params)
    z, (x0, a1, h1, a2, h2, a3, h3) = forward(params, x)
    n = x.shape[0]
    L = float(np.mean(pos_weight * y * softplus(-z) + (1.0 - y) * softplus(z)))
    s = sigmoid(z)
    d4 = (pos_weight * y * (s - 1.0) + (1.0 - y) * s) / n          # dL/dz
    g = np.zeros_like(params)
    gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4 = split(g)
    gW4[:] = d4 @ h3
    gb4[0] = d4.sum()
    d3 = np.outer(d4, W4) * silu_grad(a3)
    gW3[:] = d3.T @ h2
    gb3[:] = d3.sum(axis=0)
    d2 = (d3 @ W3) * silu_grad(a2)
    gW2[:] = d2.T @ h1
    gb2[:] = d2.sum(axis=0)
    d1 = (d2 @ W2) * silu_grad(a1)
    gW1[:] = d1.T @ x0
    gb1[:] = d1.sum(axis=0)
    return L, g


def adam_step(params, m, v, g, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1, bias-corrected); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def top_candidates(score: np.ndarray, k: int) -> np.ndarray:
    """The k highest scores (the lower grid index first among equal scores),
    returned in ascending grid order."""
    order = sorted(range(len(score)), key=lambda i: (-score[i], i))
    return np.array(sorted(order[:k]), dtype=np.int64)
