"""The slab decomposition along t (Sec. 5.2) on CPU ranks: index maps and
halo ranges bit for bit, and D_oe, D_eo, M_ee and a CG over the split
against the single-domain oracle, with two and four gloo ranks (the local operator on
each rank is the oracle's hop on its padded lattice; the decomposition's own
code does the partitioning, the halo exchange and the reductions)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1106_5673_gb300 import slab, synth  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (4, 2, 4, 8)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 4])
def test_index_maps_and_slices(world):
    """Every global site has exactly one owner, the local <-> global maps
    invert each other, and the per-rank slices of fields tile the global ones."""
    V = int(np.prod(DIMS))
    lex = np.arange(V)
    owners = slab.SlabLayout(DIMS, world, 0).owner_of_global_lex(lex)
    assert np.array_equal(np.bincount(owners, minlength=world), np.full(world, V // world))
    v = np.arange(V // 2 * 3).reshape(V // 2, 3)
    U = np.arange(4 * V * 9).reshape(4, V, 3, 3)
    parts_v, parts_U = [], []
    for r in range(world):
        L = slab.SlabLayout(DIMS, world, r)
        loc = np.arange(L.S * L.lt)
        g = L.local_to_global_lex(loc)
        assert np.array_equal(L.global_to_local_lex(g), loc)
        assert np.all(L.owner_of_global_lex(g) == r)
        parts_v.append(L.take_local_vector(v))
        parts_U.append(L.take_local_links(U))
        # the padded field carries the slab at [S, S + Vh_loc)
        pv = L.pad_vector(parts_v[-1], np.full((L.S // 2, 3), -1), np.full((L.S // 2, 3), -2))
        assert np.array_equal(L.interior(pv), parts_v[-1])
        assert pv.shape[0] == L.Vh_pad and np.all(pv[:L.S // 2] == 0) and np.all(pv[L.S // 2:L.S] == -1)
    assert np.array_equal(np.concatenate(parts_v), v)
    assert np.array_equal(np.concatenate(parts_U, axis=1), U)


def test_uneven_split_rejected():
    with pytest.raises(ValueError):
        slab.SlabLayout((4, 4, 4, 6), 2, 0)  # slabs of 3 slices would change the parity of sites
    with pytest.raises(ValueError):
        slab.SlabLayout((4, 4, 4, 8), 3, 0)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        U = synth.haar_links(DIMS, 7)
        x = synth.gaussian_vector(DIMS, 8)
        L = slab.SlabLayout(DIMS, world, rank)
        op = slab.SlabOperator(L, slab.TorchComm(dist), lambda d, Up, par, v: O.dslash(d, Up, par, v),
                               L.take_local_links(U))
        # the link halos are the neighbouring slices of the global field, bit for bit
        S, lt = L.S, L.lt
        below = (L.t0 - 1) % DIMS[3]
        above = (L.t0 + lt) % DIMS[3]
        halo_ok = (np.array_equal(op.link_halos[0], U[:, below * S:(below + 1) * S])
                   and np.array_equal(op.link_halos[1], U[:, above * S:(above + 1) * S]))
        xl = L.take_local_vector(x)
        res = {"halo_ok": halo_ok,
               "doe": op.dslash(1, xl), "deo": op.dslash(0, xl), "M": op.apply_M(0.1, xl)}
        xs, it = op.cg(0.1, 0.02, xl, tol=1e-30, maxit=25)
        res["cg"] = xs
        res["cg_iters"] = it
        res["dot"] = op.dot(xl, xl)
        q.put((rank, res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_match_the_single_domain_oracle(world):
    """Two ranks (each rank's lower and upper neighbour is the same rank)
    and four (all different), slabs of 4 and 2 time slices."""
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    U = synth.haar_links(DIMS, 7)
    x = synth.gaussian_vector(DIMS, 8)

    def cat(key):
        return np.concatenate([res[r][key] for r in range(world)])

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    assert all(res[r]["halo_ok"] for r in range(world))
    assert rel(cat("doe"), O.dslash(DIMS, U, 1, x)) < 1e-14
    assert rel(cat("deo"), O.dslash(DIMS, U, 0, x)) < 1e-14
    assert rel(cat("M"), O.apply_M(DIMS, U, 0.1, x)) < 1e-14
    assert abs(res[0]["dot"] - np.vdot(x, x).real) < 1e-13 * np.vdot(x, x).real
    # 25 CG iterations over the split and on the single domain (the oracle's CG)
    xo, it, _ = O.cg(DIMS, U, 0.1, 0.02, x, tol=1e-30, maxit=25)
    assert res[0]["cg_iters"] == it == 25
    assert rel(cat("cg"), xo) < 1e-12
