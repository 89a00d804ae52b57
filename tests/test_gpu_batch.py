"""GPU parity of the batched hop: several lattices of different sizes, many
right-hand sides each, one launch; every output against the FP64 oracle's
D_eo / D_oe (FP32 tolerance 2e-6, BF16 links 2e-2)."""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), 3), ((6, 4, 6, 10), 5), ((8, 8, 8, 8), 2)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _setup(S, seed):
    lats, Us, xs = [], [], []
    for i, (dims, nr) in enumerate(CASES):
        U = synth.near_unit_links(dims, 0.5, seed + i)
        L = S.Lattice(dims)
        L.load_gauge(U)
        x = np.stack([synth.gaussian_vector(dims, 100 * seed + 10 * i + j) for j in range(nr)])
        lats.append(L)
        Us.append(U)
        xs.append(x)
    return lats, Us, xs


@pytest.mark.parametrize("out_par", [0, 1])
@pytest.mark.parametrize("prec,tol", [(1, 2e-6), (2, 2e-2)])
def test_batched_hop_matches_oracle(S, out_par, prec, tol):
    lats, Us, xs = _setup(S, 3 + out_par)
    ins = [torch.from_numpy(x).cuda().to(torch.complex64).contiguous() for x in xs]
    outs, cfg = S.dslash_batch(lats, ins, out_par=out_par, prec=prec)
    assert cfg[0] in (64, 128, 256) and cfg[1] in (1, 2, 4, 8)
    torch.cuda.synchronize()
    for (dims, nr), U, x, y in zip(CASES, Us, xs, outs):
        y = y.cpu().numpy()
        for j in range(nr):
            ref = O.dslash(dims, U, out_par, x[j])
            err = rel(y[j], ref)
            assert err < tol, (dims, j, err)
            if prec == 2:
                assert err > 1e-5


@pytest.mark.parametrize("shape", ["128,4,0,0", "128,4,1,0", "128,4,0,1", "128,4,1,1", "64,8,1,1", "256,2,0,1",
                                   "64,1,0,1"])
def test_batched_hop_every_launch_shape(S, monkeypatch, shape):
    """Every launch shape the tuner can choose (block size, right-hand sides
    per thread, persistent grid or one block per tile, site blocks or
    right-hand-side groups fastest) gives the oracle's hop."""
    monkeypatch.setenv("STAG_BATCH_CFG", shape)
    lats, Us, xs = _setup(S, 7)
    ins = [torch.from_numpy(x).cuda().to(torch.complex64).contiguous() for x in xs]
    outs, cfg = S.dslash_batch(lats, ins, out_par=1, prec=1)
    assert list(cfg) == [int(v) for v in shape.split(",")[:2]]
    torch.cuda.synchronize()
    for (dims, nr), U, x, y in zip(CASES, Us, xs, outs):
        y = y.cpu().numpy()
        for j in range(nr):
            assert rel(y[j], O.dslash(dims, U, 1, x[j])) < 2e-6, (shape, dims, j)


def test_batched_hop_in_cuda_graph(S):
    """After the first (tuning) call the launch is capturable: a CUDA graph
    replayed on new inputs gives the oracle's results."""
    lats, Us, xs = _setup(S, 7)
    ins = [torch.from_numpy(x).cuda().to(torch.complex64).contiguous() for x in xs]
    outs, _ = S.dslash_batch(lats, ins, out_par=1)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            S.dslash_batch(lats, ins, outs, out_par=1)
    torch.cuda.current_stream().wait_stream(s)
    xs2 = [x[::-1].copy() for x in xs]
    for buf, x in zip(ins, xs2):
        buf.copy_(torch.from_numpy(x).to(torch.complex64))
    g.replay()
    torch.cuda.synchronize()
    for (dims, nr), U, x, y in zip(CASES, Us, xs2, outs):
        y = y.cpu().numpy()
        for j in range(nr):
            assert rel(y[j], O.dslash(dims, U, 1, x[j])) < 2e-6


def test_batched_hop_argument_errors(S):
    lats, _, xs = _setup(S, 9)
    ins = [torch.from_numpy(x).cuda().to(torch.complex64).contiguous() for x in xs]
    with pytest.raises(ValueError):
        S.dslash_batch(lats, [ins[1], ins[0], ins[2]])
    with pytest.raises(S.StagError):
        S.dslash_batch(lats, ins, out_par=2)
