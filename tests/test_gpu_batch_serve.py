"""Batched and served forms on the GPU: a scenario's result is the same alone, in
a batch graph, and in the server's mix (bit-identical: no cross-scenario
interaction, deterministic kernels)."""
import os

import numpy as np
import pytest

from workloads import scenarios as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1661_gb300 import build
    build.build()


def _mix():
    return [sc.tsunami(nx=40, ny=10, N=3, nlevels=4, amp=1.5, src=(150e3, 40e3)),
            sc.tsunami(nx=24, ny=8, N=4, nlevels=3, amp=3.0, src=(100e3, 60e3)),
            sc.dam_break(nx=40, ny=4, N=3),
            sc.hump_square(n=12, N=2)]


@pytest.mark.parametrize("precision", ["fp32tc", "fp64"])
def test_batch_graph_equals_solvers_alone(precision):
    import paper_1403_1661_gb300 as P
    alone = [P.solver_from_scenario(s, precision=precision) for s in _mix()]
    mixed = [P.solver_from_scenario(s, precision=precision) for s in _mix()]
    for s in alone:
        s.step(3)
    b = P.Batch(mixed)
    b.step(3)
    for a, m in zip(alone, mixed):
        xa, xm = a.get_state(), m.get_state()
        for u, v in zip(xa[:3], xm[:3]):
            assert np.array_equal(u, v)
        assert xa[3] == xm[3]
        assert a.stats()["dof_updates"] == m.stats()["dof_updates"]
    b.close()


def test_batch_uneven_macro_counts_equal_alone():
    """One batch step advances each scenario by its own number of macro steps
    (n_macro_each = 0, 1, 2, 3): every result equals the same solver stepped alone
    that many macro steps, bit for bit, and a count of 0 leaves a solver untouched."""
    import paper_1403_1661_gb300 as P
    counts = [2, 0, 3, 1]
    alone = [P.solver_from_scenario(s, precision="fp32tc") for s in _mix()]
    mixed = [P.solver_from_scenario(s, precision="fp32tc") for s in _mix()]
    for s, c in zip(alone, counts):
        if c:
            s.step(c)
    b = P.Batch(mixed, max_macro=3)
    st = b.step(counts)
    assert (st == 0).all()
    for a, m in zip(alone, mixed):
        xa, xm = a.get_state(), m.get_state()
        for u, v in zip(xa[:3], xm[:3]):
            assert np.array_equal(u, v)
        assert xa[3] == xm[3]
        assert a.stats()["dof_updates"] == m.stats()["dof_updates"]
    assert b.launches() == 2 * 3   # two kernels per (tier, order) group: N = 3, 4, 2
    b.close()


def test_batch_held_scenario_times_out_and_the_rest_complete():
    """The bounded device wait: scenario 1's release is withheld (swe_batch_hold), so
    its first phase waits until the 50 ms wait limit and gives up; the step reports
    SWE_ETIMEOUT for it alone, its state and time are untouched, the other scenarios
    complete and equal their solvers run alone. Released again, it steps normally.
    Nothing faults: the kernel's wait ends on a time bound and it returns."""
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    alone = [P.solver_from_scenario(s, precision="fp32tc") for s in _mix()]
    mixed = [P.solver_from_scenario(s, precision="fp32tc") for s in _mix()]
    before = mixed[1].get_state()
    b = P.Batch(mixed, max_macro=2)
    b.set_wait_limit(0.05)
    b.hold(1)
    st = b.step(2, check=False)
    assert st.tolist() == [0, nat.SWE_ETIMEOUT, 0, 0]
    after = mixed[1].get_state()
    for u, v in zip(before, after):
        assert np.array_equal(np.asarray(u), np.asarray(v))
    for i in (0, 2, 3):
        alone[i].step(2)
        for u, v in zip(alone[i].get_state()[:3], mixed[i].get_state()[:3]):
            assert np.array_equal(u, v)
    b.hold(1, False)
    st = b.step([0, 2, 0, 0])
    assert (st == 0).all()
    alone[1].step(2)
    for u, v in zip(alone[1].get_state()[:3], mixed[1].get_state()[:3]):
        assert np.array_equal(u, v)
    b.close()


def test_served_results_equal_alone():
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300.serve import GpuFactory, Request, Server
    scns = _mix()
    reqs = [Request(rid=i, arrival=0.002 * i, scenario=s, substeps=24) for i, s in enumerate(scns)]
    srv = Server(budget_bytes=2e9, max_slots=3, macro_per_round=1, factory=GpuFactory("fp32tc", keep_state=True),
                 start_workers=2)
    out = srv.run(reqs)
    assert out["requests"] == len(scns) and out["p99_s"] >= out["p50_s"] > 0
    for r in out["done"]:
        s = P.solver_from_scenario(r.scenario, precision="fp32tc")
        L = s.level_info()[0]
        s.step(-(-r.substeps // 2 ** (L - 1)))
        ref = s.get_state()
        for u, v in zip(ref[:3], r.result[:3]):
            assert np.array_equal(u, v)


def test_autotuner_and_launch_config_do_not_change_results():
    import paper_1403_1661_gb300 as P
    from paper_1403_1661_gb300 import _native as nat
    from paper_1403_1661_gb300 import batch
    before = open(batch.CACHE).read() if os.path.exists(batch.CACHE) else None
    best = P.tune(3, "fp32tc", candidates=((1, 4), (0, 2), (0, 8)), reps=1, force=True)
    assert (best["ctas_per_sm"], best["tc_warps"]) in ((1, 4), (0, 2), (0, 8))
    # a narrower search leaves the cached full-search results alone
    after = open(batch.CACHE).read() if os.path.exists(batch.CACHE) else None
    assert after == before
    scn = sc.tsunami(nx=40, ny=10, N=3, nlevels=4)
    a = P.solver_from_scenario(scn, precision="fp32tc")
    b = P.solver_from_scenario(scn, precision="fp32tc")
    b.set_launch_config(1)
    a.step(2)
    b.step(2)
    for u, v in zip(a.get_state()[:3], b.get_state()[:3]):
        assert np.array_equal(u, v)
    # warps per tensor-core CTA: every count that fits gives the same state, alone
    # and in a batch; one that does not fit is refused
    scn5 = sc.tsunami(nx=40, ny=10, N=5, nlevels=4)
    ref = P.solver_from_scenario(scn5, precision="fp32tc")
    ref.step(2)
    want = ref.get_state()[:3]
    for w in (1, 3, 7):
        c = P.solver_from_scenario(scn5, precision="fp32tc")
        c.set_tc_warps(w)
        c.step(2)
        for u, v in zip(want, c.get_state()[:3]):
            assert np.array_equal(u, v)
        d = P.solver_from_scenario(scn5, precision="fp32tc")
        d.set_launch_config({"ctas_per_sm": 0, "tc_warps": w})
        bb = P.Batch([d], max_macro=2)
        bb.step(2)
        for u, v in zip(want, d.get_state()[:3]):
            assert np.array_equal(u, v)
        bb.close()
    with pytest.raises(nat.SWEError):
        ref.set_tc_warps(8)        # 8 x 29 KB of N = 5 tiles exceed an SM's shared memory


def test_full_ensemble_batch_equals_alone_on_a_sample():
    """The batched ensemble at its full size, built as the benchmark builds it (64
    sloped-beach scenarios of 5k-200k triangles, N in {3, 4, 5}, autotuned launch
    shapes, one graph launch per macro step of all of them): after three macro
    steps, eight seeded scenarios equal the same scenarios run alone, bit for bit."""
    import paper_1403_1661_gb300 as P
    scns = sc.ensemble()
    assert len(scns) == 64
    tuned = {N: P.tune(N, "fp32tc") for N in sorted({s.N for s in scns})}
    solvers = []
    for s in scns:
        so = P.solver_from_scenario(s, precision="fp32tc")
        so.set_launch_config(tuned[s.N])
        solvers.append(so)
    b = P.Batch(solvers)
    b.step(3)
    pick = sorted(np.random.Generator(np.random.PCG64(9)).choice(len(scns), size=8, replace=False))
    for i in pick:
        a = P.solver_from_scenario(scns[i], precision="fp32tc")
        a.set_launch_config(tuned[scns[i].N])
        a.step(3)
        xa, xb = a.get_state(), solvers[i].get_state()
        assert np.isfinite(xb[0]).all() and xa[3] == xb[3]
        for u, v in zip(xa[:3], xb[:3]):
            assert np.array_equal(u, v)
        assert a.stats()["dof_updates"] == solvers[i].stats()["dof_updates"]
        a.close()
    b.close()
    for so in solvers:
        so.close()


def test_served_nonfinite_solve_is_stopped_and_the_other_completes():
    """A served solve whose state turns non-finite is stopped at the server's next
    health check and reported as failed, and the request served beside it
    completes. The failing request is the served stream's own (a 3,872-triangle
    beach at N = 2 whose thin shoreline layers outrun the levels fixed at t = 0;
    the FP64 oracle diverges on it as well): the kernels run on non-finite numbers
    and the device flag reports them, no GPU fault is involved."""
    from paper_1403_1661_gb300.serve import GpuFactory, Request, Server
    bad = sc.served_stream(duration=5.0)[19][1]
    assert bad.name == "tsunami_88x22x2_N2_L4"
    good = sc.tsunami(nx=40, ny=10, N=3, nlevels=4, amp=1.5, src=(150e3, 40e3))
    reqs = [Request(rid=0, arrival=0.0, scenario=bad, substeps=500),
            Request(rid=1, arrival=0.0, scenario=good, substeps=24)]
    srv = Server(budget_bytes=2e9, max_slots=2, macro_per_round=4, factory=GpuFactory("fp32tc"),
                 health_every=2)
    out = srv.run(reqs)
    st = {r.rid: (r.status, r.error) for r in out["done"] + out["ended"]}
    assert st[0] == ("failed", "non-finite state")
    assert st[1] == ("done", None) and out["requests"] == 1 and out["failed"] == 1
