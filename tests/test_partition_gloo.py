"""The (P, Q)-sharded build on two ranks (gloo, CPU) equals the single build.

The sharded design: every rank owns a block-cyclic share of the (P, Q) tiles
of the point-space matrices.  It forms D and the k-convolution on its tiles
only and adds M[P, Q] Psi[Q] into a partial Y.  A reduce-scatter by P sums
the partial Y and leaves each rank its own slice of the P rows; each rank
back-projects that slice and an all-reduce sums KC and E_x.  The per-rank arithmetic is the FP64 oracle's (steps 1-5 of
oracle/thc_oracle.py), so this checks the partition and the exchange steps,
not the kernels.  The exchanges carry O(N_k N_P n) values against the
O(N_k N_P^2) kernel each rank keeps."""
import os
import socket

import numpy as np
import pytest

MESH = (3, 2, 2)
TILE = 16


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from oracle import thc_oracle as O
    from paper_2304_05505_gb300 import cells

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    r = cells.random_problem(MESH, nbas=14, nocc=3, nisdf=70, seed=21)
    X, C, V = r["X"], r["C"], r["V"]
    nk, _, npt = X.shape
    Psi = O.collocate(X, C)                           # replicated (cheap, N_k N_P n)
    nt = (npt + TILE - 1) // TILE
    tiles = [(a, b) for a in range(nt) for b in range(nt)]
    mine = tiles[rank::world]                         # block-cyclic tile ownership
    Ypart = np.zeros_like(Psi)
    for (a, b) in mine:
        pr = slice(a * TILE, min(npt, (a + 1) * TILE))
        qr = slice(b * TILE, min(npt, (b + 1) * TILE))
        D = np.stack([Psi[k][pr] @ Psi[k][qr].conj().T for k in range(nk)])   # step 2 on the tile
        M = O.kconv_direct(D, V[:, pr, qr], MESH)                             # step 3 on the tile
        for k in range(nk):
            Ypart[k][pr] += M[k] @ Psi[k][qr]                                 # step 4a, partial over Q
    # reduce-scatter of Y by P: the Q-partial products are summed and each rank
    # receives only its own slice of the P rows (P-major so the slices are contiguous)
    assert npt % world == 0
    rows = slice(rank * npt // world, (rank + 1) * npt // world)
    Yp = torch.from_numpy(np.ascontiguousarray(Ypart.transpose(1, 0, 2)))
    Ymine = torch.zeros((npt // world, nk, Ypart.shape[2]), dtype=Yp.dtype)
    dist.reduce_scatter_tensor(Ymine, Yp)
    Yr = Ymine.numpy().transpose(1, 0, 2)            # [N_k][rows of this rank][n]
    KC = torch.from_numpy(np.stack([X[k][:, rows].conj() @ Yr[k] for k in range(nk)]))
    ex = torch.tensor([-np.sum(Psi[:, rows].conj() * Yr).real / nk])
    dist.all_reduce(KC)
    dist.all_reduce(ex)
    if rank == 0:
        np.save(os.path.join(out_dir, "kc.npy"), KC.numpy())
        np.save(os.path.join(out_dir, "ex.npy"), ex.numpy())
    dist.destroy_process_group()


def test_two_rank_partition_matches_single(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    from oracle import thc_oracle as O
    from paper_2304_05505_gb300 import cells

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = cells.random_problem(MESH, nbas=14, nocc=3, nisdf=70, seed=21)
    ref = O.build(r["X"], r["C"], r["V"], MESH)
    kc = np.load(tmp_path / "kc.npy")
    ex = float(np.load(tmp_path / "ex.npy")[0])
    assert np.abs(kc - ref["KC"]).max() < 1e-12 * np.abs(ref["KC"]).max()
    assert abs(ex - ref["Ex"]) < 1e-12 * abs(ref["Ex"])
