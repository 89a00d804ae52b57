"""The allocation-free M_ee entry point, for callers that must not allocate
device memory when they apply the operator (a framework that owns the device
memory pool, or a latency-critical loop that cannot afford cudaMalloc's
implicit synchronisation).

It is checked through the C ABI on two calls in a row (the calls share the
library's fixed scratch array, so the second call must not see anything of
the first) against the context-based stag_apply_M and against the FP64
oracle's M_ee, to the FP64 operator tolerance of the other parity tests
(1e-13 relative to the library, 1e-12 to the oracle).  This file is
collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 6, 10), (32, 32, 32, 8)])
def test_noalloc_M_matches_context_entry_point_on_two_calls(S, dims):
    U = synth.haar_links(dims, 51)
    L = S.Lattice(dims)
    L.load_gauge(U)
    links = torch.from_numpy(U).cuda()
    for call, mass in enumerate((0.05, 0.3)):
        x = torch.from_numpy(synth.gaussian_vector(dims, 60 + call)).cuda()
        ref = L.vector()
        L.apply_M(mass, x, ref)
        out = torch.full_like(ref, float("nan"))
        assert S.apply_M_noalloc(dims, links, mass, x, out) == S.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert _rel(got, ref.cpu().numpy()) < 1e-13, (dims, call)
        want = O.apply_M(dims, U, mass, np.ascontiguousarray(x.cpu().numpy()))
        assert _rel(got, want) < 1e-12, (dims, call)


def test_noalloc_rejects_lattices_beyond_its_scratch(S):
    dims = (64, 32, 32, 8)  # V/2 = 2^18 > 2^17
    links = torch.zeros((1,), dtype=torch.complex128, device="cuda")
    x = torch.zeros((1,), dtype=torch.complex128, device="cuda")
    y = torch.zeros((1,), dtype=torch.complex128, device="cuda")
    assert S.apply_M_noalloc(dims, links, 0.1, x, y) == S.ERR_ARG
    assert S.apply_M_noalloc((3, 4, 4, 4), links, 0.1, x, y) == S.ERR_ARG
    # extents whose product would overflow a 32-bit int, or wrap to a small
    # volume in 64 bits, are rejected before anything is launched
    assert S.apply_M_noalloc((65536, 65536, 2, 2), links, 0.1, x, y) == S.ERR_ARG
    assert S.apply_M_noalloc((1 << 30, 2, 2, 2), links, 0.1, x, y) == S.ERR_ARG
    assert S.apply_M_noalloc((-2, 4, 4, 4), links, 0.1, x, y) == S.ERR_ARG
