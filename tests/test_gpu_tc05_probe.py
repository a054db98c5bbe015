"""The volume-projection probe (Section 7.1's N(Q) = Pr cF1 + ..., one field, N = 4
shapes) on both tensor-core paths: warp-level mma.sync and tcgen05 with a TMEM
accumulator (variants: CTA barriers, an mbarrier pipeline, wider instructions that
repeat the operator's columns, and the flux stored to TMEM as the A operand). All
must equal the product written out in numpy with the same TF32 operand rounding;
the timings are printed for the design notes."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROWS, KQ, NN = 128, 40, 16


def _tf32(a):
    """Round float32 values to TF32 (10 mantissa bits), to nearest, ties away from zero."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()
    from paper_1403_1661_gb300 import _native as nat
    return torch, nat, nat.lib()


def _run(torch, nat, lib, impl, nctas, tiles, x, y, c, b, stream=None):
    d = torch.full((nctas * ROWS * NN,), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.full((nctas,), -99, dtype=torch.int32, device="cuda")
    s = stream or torch.cuda.current_stream()
    rc = lib.swe_tc_projection_probe(impl, nctas, tiles, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                     C.c_void_p(c.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(d.data_ptr()),
                                     C.c_void_p(st.data_ptr()), C.c_void_p(s.cuda_stream))
    assert rc == nat.SWE_OK, lib.swe_last_error()
    return d, st


@pytest.mark.parametrize("tiles", [1, 2, 5, 11])
def test_projection_probe_both_paths_match_numpy(tiles):
    torch, nat, lib = _setup()
    rng = np.random.Generator(np.random.PCG64(11 + tiles))
    nctas = 3
    x = rng.uniform(-1, 1, nctas * tiles * ROWS).astype(np.float32)
    y = rng.uniform(-1, 1, nctas * tiles * ROWS).astype(np.float32)
    c = rng.uniform(-1, 1, KQ).astype(np.float32)
    b = rng.uniform(-1, 1, (KQ, NN)).astype(np.float32)
    # the flux a[e][q] = fl(x[e] c[q] + y[e]) (one rounding, as the kernels' fmaf), then TF32
    a = _tf32((x.astype(np.float64)[:, None] * c[None, :] + y[:, None]).astype(np.float32))
    bt = _tf32(b).astype(np.float64)
    a3 = a.astype(np.float64).reshape(nctas, tiles, ROWS, KQ)
    want = np.einsum("ctrq,qn->crn", a3, bt)
    scale = np.einsum("ctrq,qn->crn", np.abs(a3), np.abs(bt))
    dx, dy, dc, db = (torch.from_numpy(v).cuda() for v in (x, y, c, b.reshape(-1)))
    got = {}
    for impl in (0, 1, 2, 3, 4, 5):
        d, st = _run(torch, nat, lib, impl, nctas, tiles, dx, dy, dc, db)
        torch.cuda.synchronize()
        got[impl] = d.cpu().numpy().astype(np.float64).reshape(nctas, ROWS, NN)
        if impl > 0:
            assert (st.cpu().numpy() == nat.SWE_OK).all()
        err = np.abs(got[impl] - want) / scale
        # FP32 accumulation of at most 5 x 40 products: a few units of 2^-24 of the
        # sum of magnitudes; 1e-5 leaves room for the accumulation order only
        assert err.max() < 1e-5, (impl, float(err.max()))
    print(f"PARITY tc05 projection tiles={tiles}: max |mma.sync - tcgen05| / sum|ab| "
          f"{float((np.abs(got[0] - got[1]) / scale).max()):.2e}, pipelined "
          f"{float((np.abs(got[0] - got[2]) / scale).max()):.2e}, N = 64 / 128 "
          f"{float((np.abs(got[0] - got[3]) / scale).max()):.2e} / "
          f"{float((np.abs(got[0] - got[4]) / scale).max()):.2e}, A in TMEM "
          f"{float((np.abs(got[0] - got[5]) / scale).max()):.2e}", flush=True)


def test_projection_probe_timing():
    torch, nat, lib = _setup()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = 256
    rng = np.random.Generator(np.random.PCG64(5))
    c = torch.from_numpy(rng.uniform(-1, 1, KQ).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.uniform(-1, 1, KQ * NN).astype(np.float32)).cuda()
    res = {}
    for per_sm in (2, 4):
        nctas = nsm * per_sm
        x = torch.rand(nctas * tiles * ROWS, device="cuda")
        y = torch.rand(nctas * tiles * ROWS, device="cuda")
        for impl in (0, 1, 2, 3, 4, 5):
            if per_sm > 2 and impl in (2, 4):
                continue   # 83 KB / 61 KB of shared memory per CTA: at most two / three per SM
            for _ in range(3):
                _run(torch, nat, lib, impl, nctas, tiles, x, y, c, b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record()
            for _ in range(reps):
                d, st = _run(torch, nat, lib, impl, nctas, tiles, x, y, c, b)
            e1.record()
            torch.cuda.synchronize()
            if impl > 0:
                assert (st.cpu().numpy() == nat.SWE_OK).all()
            ms = e0.elapsed_time(e1) / reps
            rows = nctas * tiles * ROWS
            res[(per_sm, impl)] = ms
            name = ("mma.sync", "tcgen05 (CTA barriers)", "tcgen05 (4-stage mbarrier pipeline)",
                    "tcgen05 N = 64 (4x the columns)", "tcgen05 N = 128 (8x the columns)",
                    "tcgen05, A stored to TMEM")[impl]
            print(f"TIMING tc05 projection {per_sm} CTAs/SM {name}: "
                  f"{ms:.3f} ms for {rows} rows, {rows / ms / 1e6:.2f} G rows/s, "
                  f"{2.0 * rows * KQ * NN / ms / 1e9:.1f} TFLOP/s (TF32)", flush=True)
    assert all(v > 0 for v in res.values())
