"""The x-slab decomposition of one solve (paper_2605_04735_gb300.slab) on CPU
ranks: gloo process groups of 2 and 3 ranks, each rank applying the oracle's
FP64 matrix-free operator to its own slab (owned node planes plus one ghost
plane per neighbour, filled by the halo exchange).  The distributed K u and
the distributed Jacobi-PCG iterates must reproduce the one-rank results (the
only difference is the order of the dot products' partial sums)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import fem
from oracle import fullsize as FS
from paper_2605_04735_gb300 import inputs as I
from paper_2605_04735_gb300 import slab as SL

NX, NY, NZ = 13, 4, 3
ITERS = 25


def _problem():
    rho = I.density_uniform(NX, NY, NZ, 0.05, 1.0, 77)
    P = fem.Problem(NX, NY, NZ, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, rho)
    return P


def _local_operator(P, s):
    """apply_local, D^-1, f and the fixed mask of rank s's slab, from the
    oracle's operator on the local grid of element layers [e_lo, e_hi)."""
    g = fem.Grid(s.e_hi - s.e_lo, NY, NZ)
    E = s.local_elements(P.E)
    shape = (s.n_local_planes, NZ + 1, NY + 1, 3)

    def apply_local(u):
        flat = np.ascontiguousarray(u.transpose(1, 2, 0, 3)).reshape(-1)
        y = FS.apply(g, E, P.k0, flat)
        return np.ascontiguousarray(y.reshape(NZ + 1, NY + 1, s.n_local_planes, 3)
                                    .transpose(2, 0, 1, 3))

    diag = fem.assemble(g, E, P.k0).diagonal()
    diag = np.ascontiguousarray(diag.reshape(NZ + 1, NY + 1, s.n_local_planes, 3)
                                .transpose(2, 0, 1, 3))
    fixed = s.to_local(P.fixed.astype(np.float64)) > 0.5
    dinv = np.where(fixed | (diag <= 0), 0.0, 1.0 / np.where(diag > 0, diag, 1.0))
    f = s.to_local(P.f)
    assert f.shape == shape
    return apply_local, dinv, f, fixed


def _run(s, comm, P, u_global):
    apply_local, dinv, f, fixed = _local_operator(P, s)
    u = s.to_local(u_global)
    u[s.owned.start:s.owned.stop] = u[s.owned]  # owned planes from the global vector
    if s.left is not None:
        u[0] = 0.0
    if s.right is not None:
        u[-1] = 0.0                              # ghosts come only from the exchange
    comm.exchange(u)
    y = apply_local(u)
    y_all = comm.allgather_planes(y[s.owned], NX + 1)
    iterates = []
    x, it, rel = SL.jacobi_pcg(s, comm, apply_local, dinv, f, fixed, rtol=0.0, maxiter=ITERS,
                               record=iterates)
    full = [comm.allgather_planes(xi, NX + 1) for xi in iterates]
    return y_all, full


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        P = _problem()
        u = np.random.default_rng(3).normal(size=P.grid.n_dof)
        u[P.fixed] = 0.0
        s = SL.Slab.make(NX, NY, NZ, ws, rank)
        y, its = _run(s, SL.Comm(s), P, u)
        out[rank] = (y, np.stack(its))
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_node_plane_once_with_matching_ghosts():
    for world in (1, 2, 3, 5):
        slabs = [SL.Slab.make(NX, NY, NZ, world, r) for r in range(world)]
        owned = np.concatenate([np.arange(s.i0, s.i1) for s in slabs])
        assert np.array_equal(owned, np.arange(NX + 1))
        for a, b in zip(slabs, slabs[1:]):
            assert a.hi == b.i0 and b.lo == a.i1 - 1  # each ghost is the neighbour's owned plane
        for s in slabs:  # every element touching an owned node is held locally
            assert s.e_lo <= max(s.i0 - 1, 0) and s.e_hi >= min(s.i1, NX)
    g = np.arange(3 * (NX + 1) * (NY + 1) * (NZ + 1), dtype=float)
    back = np.zeros_like(g)
    for r in range(3):
        s = SL.Slab.make(NX, NY, NZ, 3, r)
        s.from_local(s.to_local(g), out=back)
    assert np.array_equal(back, g)
    with pytest.raises(ValueError):
        SL.split_planes(2, 3)


def test_coarse_levels_below_the_threshold_are_gathered():
    lv = SL.coarse_slabs(192, 96, 96, 4, 6, gather_below=4096)
    assert [l["grid"] for l in lv][:3] == [(192, 96, 96), (96, 48, 48), (48, 24, 24)]
    assert not lv[0]["gathered"] and lv[-1]["gathered"]
    assert all(l["gathered"] for l in lv if l["nodes"] < 4096)
    for l in lv:
        if not l["gathered"]:
            assert l["split"][-1][1] == l["grid"][0] + 1


def test_one_rank_matches_the_oracle_operator_and_cg():
    P = _problem()
    u = np.random.default_rng(3).normal(size=P.grid.n_dof)
    u[P.fixed] = 0.0
    s = SL.Slab.make(NX, NY, NZ, 1, 0)
    y, its = _run(s, SL.LocalComm(s), P, u)
    ref = FS.apply(P.grid, P.E, P.k0, u)
    assert np.allclose(s.from_local(y, owned_only=False), ref, rtol=0, atol=1e-13 * abs(ref).max())
    # the CG converges to the direct solution (the driver is a plain Jacobi-PCG)
    apply_local, dinv, f, fixed = _local_operator(P, s)
    x, it, rel = SL.jacobi_pcg(s, SL.LocalComm(s), apply_local, dinv, f, fixed, rtol=1e-12)
    u_ref = P.solve()
    assert rel <= 1e-12
    assert np.linalg.norm(s.from_local(x) - u_ref) <= 1e-8 * np.linalg.norm(u_ref)


@pytest.mark.parametrize("ws", [2, 3])
def test_gloo_ranks_reproduce_the_one_rank_operator_and_cg_iterates(ws):
    P = _problem()
    u = np.random.default_rng(3).normal(size=P.grid.n_dof)
    u[P.fixed] = 0.0
    s1 = SL.Slab.make(NX, NY, NZ, 1, 0)
    y1, its1 = _run(s1, SL.LocalComm(s1), P, u)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(ws):
        y, its = res[r]
        # K u: the same element sums on every owned node (their order may differ
        # with the parity of a slab's first element: rounding only)
        assert np.abs(y - y1).max() <= 1e-14 * np.abs(y1).max()
        # CG iterates: dot products summed from ws partials, so equal to rounding
        assert its.shape == np.stack(its1).shape
        for k in range(ITERS):
            d = np.linalg.norm(its[k] - its1[k]) / np.linalg.norm(its1[k])
            assert d <= 1e-11, (r, k, d)
