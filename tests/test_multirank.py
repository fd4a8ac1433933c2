"""The multi-process path on CPU (world size 2, gloo).

FTLM shards over independent random vectors: rank k runs vectors
k*R .. k*R+R-1 of the same Philox stream (vec_offset), and the thermodynamics
of the whole set follow from gathering the per-vector tridiagonal data and
one call of the host-only ftlm_sums (the merge needs the common E0, which
ftlm_sums takes over all gathered vectors).  Here the per-rank Lanczos runs
come from the oracle (no GPU on this machine); the sharding, the gather and
the library's merge are what is under test."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

import ftlm_workloads as W

R_LOCAL, M = 3, 25


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    import paper_2607_25585_gb300 as F

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.ring(N=5, two_s=2)
    s = oracle.System(**{k: v for k, v in w.items() if k != "name"})
    T = W.temperatures()
    o = oracle.ftlm(s, R=R_LOCAL, M=M, T=T, seed=4, vec_offset=rank * R_LOCAL)
    parts = [None] * world
    dist.all_gather_object(parts, {k: o[k] for k in ("alpha", "beta", "p", "M_eff")})
    if rank == 0:
        cat = {k: np.concatenate([p[k] for p in parts]) for k in ("alpha", "beta", "p", "M_eff")}
        merged = F.sums(cat["alpha"], cat["beta"], cat["p"], cat["M_eff"], s.dim, s.g, T)
        np.savez(out_path, **{k: merged[k] for k in ("lnZ", "E", "C", "M_B")})
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_one_process():
    import oracle
    import paper_2607_25585_gb300 as F

    oracle.build()
    F.build()
    world = 2
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "merged.npz")
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        merged = np.load(out)
        w = W.ring(N=5, two_s=2)
        s = oracle.System(**{k: v for k, v in w.items() if k != "name"})
        full = oracle.ftlm(s, R=world * R_LOCAL, M=M, T=W.temperatures(), seed=4)
        for k in ("lnZ", "E", "C", "M_B"):
            ref = full[k]
            assert np.max(np.abs(merged[k] - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())) < 1e-11, k


def _worker_sym(rank, world, port, out_path):
    """Symmetric FTLM sharded the same way: each rank gathers its vectors'
    alpha, beta, M_eff and O_ij = <v_i|u.S|v_j>; rank 0 merges with the
    host-only ftlm_sums_sym (common E0 over all vectors)."""
    import torch.distributed as dist

    import oracle
    import paper_2607_25585_gb300 as F

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.ring(N=5, two_s=2)
    s = oracle.System(**{k: v for k, v in w.items() if k != "name"})
    T = W.temperatures()
    o = oracle.sftlm(s, R=R_LOCAL, M=M, T=T, seed=4, vec_offset=rank * R_LOCAL, start="pairs")
    parts = [None] * world
    dist.all_gather_object(parts, {k: o[k] for k in ("alpha", "beta", "O", "M_eff")})
    if rank == 0:
        cat = {k: np.concatenate([p[k] for p in parts]) for k in ("alpha", "beta", "O", "M_eff")}
        mb, _ = F.sums_sym(cat["alpha"], cat["beta"], cat["O"], cat["M_eff"], s.g, T)
        np.savez(out_path, M_B_sym=mb)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_symmetric_estimator():
    import oracle
    import paper_2607_25585_gb300 as F

    oracle.build()
    F.build()
    world = 2
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "merged_sym.npz")
        mp.spawn(_worker_sym, args=(world, _free_port(), out), nprocs=world, join=True)
        merged = np.load(out)["M_B_sym"]
        w = W.ring(N=5, two_s=2)
        s = oracle.System(**{k: v for k, v in w.items() if k != "name"})
        full = oracle.sftlm(s, R=world * R_LOCAL, M=M, T=W.temperatures(), seed=4, start="pairs")["M_B_sym"]
        assert np.max(np.abs(merged - full) / np.maximum(np.abs(full), 1e-6 * np.abs(full).max())) < 1e-11
