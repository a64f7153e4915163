"""The slab partition of the operator apply on 2 gloo ranks (CPU): halo exchange of node planes and
pressure layers, the local apply on each rank's sub-mesh with its two ghost element layers, and
the owned parts of the result, against the global apply (1e-12), on the brick and on a mapped mesh
(each rank assembling from its local planes of the node coordinates).  The local applies here are
the oracle's assembled matrices on the sub-meshes (the same matrices the CUDA kernels apply); dot
products over owned nodes reduce to the global ones."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

NX, NY, NZ, K = 3, 2, 6, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(mapped):
    """Global mesh, node coordinates (moved interior vertices when mapped), viscosity, inputs."""
    from oracle import mesh as M
    from paper_1607_03936_gb300 import inputs
    mg = M.Mesh(NX, NY, NZ, K)
    X = mg.node_coords()
    if mapped:
        X = inputs.deform_vertices(X, (NX, NY, NZ), (1.0, 1.0, 1.0), 0.12, 9)
    mu = 1.0 + X[:, 0] + 2.0 * X[:, 2] ** 2
    rng = np.random.default_rng(5)
    return mg, X, mu, rng.standard_normal(mg.n_u), rng.standard_normal(mg.n_p)


def _operators(mesh, X, mu, mapped):
    """A and B of the oracle: the brick's, or the mapped mesh's with nodal coordinates X."""
    from oracle import mapped as mpd
    from oracle import operators as op
    if mapped:
        return mpd.assemble_A(mesh, X, op.point_values(mesh, mu)), mpd.assemble_B(mesh, X)
    return op.assemble_A(mesh, op.point_values(mesh, mu)), op.assemble_B(mesh)


def _worker(rank, world, port, out, mapped=False):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import mesh as M
    from paper_1607_03936_gb300 import partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mg, X, mu, u, p = _problem(mapped)
        part = partition.SlabPartition(NX, NY, NZ, K, world, rank)
        u_loc = part.local_from_global(torch.tensor(u), 3).clone()
        p_loc = part.local_pressure_from_global(torch.tensor(p), mg.Np).clone()
        # ghosts start as garbage: the halo exchange must overwrite them
        lo, hi = part.owned_local_planes()
        v = u_loc.reshape(3, part.ext_planes, part.plane)
        v[:, :lo] = 1e3
        v[:, hi:] = 1e3
        pv = p_loc.reshape(part.ext_nz, -1)
        pv[: part.z0 - part.e0] = 1e3
        pv[part.z1 - part.e0:] = 1e3
        ms = M.Mesh(NX, NY, part.ext_nz, K, 1.0, 1.0, part.ext_nz / NZ)
        mu_loc = part.local_from_global(torch.tensor(mu), 1).numpy()
        X_loc = part.local_from_global(torch.tensor(np.ascontiguousarray(X.T).ravel()), 3).reshape(3, -1).T.numpy()
        A, B = _operators(ms, X_loc, mu_loc, mapped)

        def local_apply(ul, pl):
            a, b = ul.numpy(), pl.numpy()
            return torch.tensor(A @ a + B.T @ b), torch.tensor(B @ a)

        yu, yp = partition.partitioned_apply(part, u_loc, p_loc, local_apply, mg.Np)
        d = part.dot(u_loc, u_loc, 3).item()
        out.put((rank, part.owned_planes(), yu.numpy().copy(), (part.z0, part.z1), yp.numpy().copy(), d))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mapped", [False, True])
def test_partitioned_K_apply_matches_global_on_two_gloo_ranks(mapped):
    """Brick, and a mapped mesh whose ranks assemble their sub-mesh operators from their local
    planes of the global node coordinates."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out, mapped)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted([out.get(timeout=180) for _ in range(2)], key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    sys.path.insert(0, ROOT)
    mg, X, mu, u, p = _problem(mapped)
    A, B = _operators(mg, X, mu, mapped)
    yu = (A @ u + B.T @ p).reshape(3, mg.NZ, mg.NX * mg.NY)
    yp = (B @ u).reshape(NZ, NX * NY * mg.Np)
    got_u = np.concatenate([r[2] for r in res], axis=1)
    got_p = np.concatenate([r[4] for r in res], axis=0)
    assert [r[1] for r in res] == [(0, 6), (6, 13)]
    np.testing.assert_allclose(got_u, yu, rtol=0, atol=1e-12 * np.abs(yu).max())
    np.testing.assert_allclose(got_p, yp, rtol=0, atol=1e-12 * np.abs(yp).max())
    for r in res:
        np.testing.assert_allclose(r[5], u @ u, rtol=1e-13)


def test_slab_bounds_and_ghost_layers():
    sys.path.insert(0, ROOT)
    from paper_1607_03936_gb300 import partition
    parts = [partition.SlabPartition(4, 4, 10, 2, 3, r) for r in range(3)]
    assert [(q.z0, q.z1) for q in parts] == [(0, 4), (4, 7), (7, 10)]
    assert [(q.e0, q.e1) for q in parts] == [(0, 6), (2, 9), (5, 10)]
    # owned planes tile the global planes 0..k nz exactly once
    planes = [q.owned_planes() for q in parts]
    assert planes == [(0, 8), (8, 14), (14, 21)]
    with pytest.raises(ValueError):
        partition.SlabPartition(4, 4, 5, 2, 3, 0)


def _solve_worker(rank, world, port, out, mapped=False):
    """The distributed FGMRES of partition.py on `world` gloo ranks (world 1: no process group)."""
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import mesh as M
    from paper_1607_03936_gb300 import partition
    if world > 1:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mg, X, mu, _, _ = _problem(mapped)
        part = partition.SlabPartition(NX, NY, NZ, K, world, rank)
        ms = M.Mesh(NX, NY, part.ext_nz, K, 1.0, 1.0, part.ext_nz / NZ)
        mu_loc = part.local_from_global(torch.tensor(mu), 1).numpy()
        X_loc = part.local_from_global(torch.tensor(np.ascontiguousarray(X.T).ravel()), 3).reshape(3, -1).T.numpy()
        A, B = _operators(ms, X_loc, mu_loc, mapped)

        def local_apply(ul, pl):
            a, b = ul.numpy(), pl.numpy()
            return torch.tensor(A @ a + B.T @ b), torch.tensor(B @ a)

        K_op = partition.SlabOperator(part, local_apply, mg.Np)
        b_glob = _consistent_rhs(mg, X, mu, mapped)
        lo, hi = part.owned_planes()
        bu = torch.tensor(b_glob[: mg.n_u]).reshape(3, mg.NZ, mg.NX * mg.NY)[:, lo:hi].reshape(-1)
        bp = torch.tensor(b_glob[mg.n_u:]).reshape(NZ, -1)[part.z0: part.z1].reshape(-1)
        x, its, rel = partition.fgmres(K_op, torch.cat([bu, bp]), restart=20, maxit=40, rtol=1e-14)
        out.put((rank, x[: K_op.n_u].numpy().copy(), x[K_op.n_u:].numpy().copy(), its, rel))
    finally:
        if world > 1:
            dist.destroy_process_group()


def _consistent_rhs(mg, X, mu, mapped):
    A, B = _operators(mg, X, mu, mapped)
    rng = np.random.default_rng(9)
    u = rng.standard_normal(mg.n_u) * np.tile(~mg.boundary_node_mask(), 3)
    p = rng.standard_normal(mg.n_p)
    return np.concatenate([A @ u + B.T @ p, B @ u])


def _gather(res, mg):
    u = np.concatenate([r[1].reshape(3, -1, mg.NX * mg.NY) for r in res], axis=1).reshape(-1)
    p = np.concatenate([r[2] for r in res])
    return np.concatenate([u, p])


@pytest.mark.parametrize("mapped", [False, True])
def test_partitioned_fgmres_matches_one_rank_and_oracle(mapped):
    """40 FGMRES iterations (restart 20, identity preconditioner) of the Stokes system on 2 gloo ranks
    against the same code on 1 rank and against the oracle's FGMRES on the assembled global matrices
    (brick, and a mapped mesh)."""
    import queue
    from oracle import krylov
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, out, mapped)) for r in range(2)]
    for pr in procs:
        pr.start()
    res2 = sorted([out.get(timeout=300) for _ in range(2)], key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    q1 = queue.Queue()
    _solve_worker(0, 1, 0, q1, mapped)
    res1 = [q1.get()]
    mg, X, mu, _, _ = _problem(mapped)
    x2, x1 = _gather(res2, mg), _gather(res1, mg)
    assert res2[0][3] == res1[0][3] == 40
    assert np.linalg.norm(x2 - x1) <= 1e-10 * np.linalg.norm(x1)
    A, B = _operators(mg, X, mu, mapped)
    Kg = lambda v: np.concatenate([A @ v[: mg.n_u] + B.T @ v[mg.n_u:], B @ v[: mg.n_u]])
    xo, its, _ = krylov.fgmres(Kg, lambda v: v, _consistent_rhs(mg, X, mu, mapped), rtol=1e-14, restart=20,
                               maxit=40)
    assert its == 40
    assert np.linalg.norm(x1 - xo) <= 1e-8 * np.linalg.norm(xo)
