"""The slab decomposition's data plane on one GPU: two ranks run as threads
of one process, each applying the library's FP64 hop to its padded local
lattice after the halo exchange (the exchange itself is host-side: no kernel
waits on another).  Their D_oe, D_eo and M_ee over the split equal the
library's operator on the whole lattice and the FP64 oracle."""
import threading

import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import slab, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


@pytest.mark.parametrize("world", [1, 2])
def test_slab_ranks_on_one_gpu(S, world):
    dims = (4, 4, 6, 8)
    U = synth.haar_links(dims, 21)
    x = synth.gaussian_vector(dims, 22)
    shared = slab.ThreadComm.shared(world)
    out = {}
    errors = []

    def rank_main(r):
        try:
            L = slab.SlabLayout(dims, world, r)
            op = slab.SlabOperator(L, slab.ThreadComm(shared, r, world), slab.gpu_local_hop(S, torch),
                                   L.take_local_links(U))
            xl = L.take_local_vector(x)
            out[r] = (op.dslash(1, xl), op.dslash(0, xl), op.apply_M(0.1, xl))
        except Exception as e:  # reported below
            errors.append(e)
            shared["barrier"].abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    doe, deo, M = (np.concatenate([out[r][i] for r in range(world)]) for i in range(3))
    Lg = S.Lattice(dims)
    Lg.load_gauge(U)
    ref = Lg.vector()
    Lg.apply_M(0.1, torch.from_numpy(x).cuda(), ref)
    torch.cuda.synchronize()

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    assert rel(M, ref.cpu().numpy()) < 1e-13
    assert rel(M, O.apply_M(dims, U, 0.1, x)) < 1e-13
    assert rel(doe, O.dslash(dims, U, 1, x)) < 1e-13
    assert rel(deo, O.dslash(dims, U, 0, x)) < 1e-13
