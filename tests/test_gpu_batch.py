"""Batched, continuously served solves (gp_batch_*): admission by device-memory
footprint, one launch per substep for all running solves of a precision,
convergence checks between ticks, and the guarantee that a solve's result is
the same alone and in any mix."""
import numpy as np
import pytest

from paper_2105_10517_gb300 import gpspin

pytestmark = pytest.mark.gpu

CHECK = 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def req_params(n, **kw):
    p = dict(nx=n, ny=n, xlen=32.0 * n / 128, ylen=32.0 * n / 128, dt=0.1 * (32.0 / 128) ** 2, c0=200.0, c2=-5.0,
             omeg=0.5, so_type=1, gamma=0.6, rabi=0.2)
    p.update(kw)
    return p


def run_batch(items, max_bytes=8 << 30, graphs=True, persist=None):
    """items: list of (params, submit kwargs); runs until all are done."""
    out = {}
    with gpspin.Batch(max_bytes, check_every=CHECK) as b:
        b.use_graphs(graphs)
        if persist is not None:
            b.set_persistent(persist)
        ids = [b.submit(p, **kw) for p, kw in items]
        for _ in range(10000):
            nr, nq = b.step()
            if nr == 0 and nq == 0:
                break
        for i in ids:
            st, steps, obs, psi = b.poll(i, fetch=True, release=True)
            out[i] = (st, steps, obs, psi)
    return [out[i] for i in ids]


def test_result_alone_equals_result_in_mix_bitwise():
    a = (req_params(96), dict(seed=11, tol=1e-300, cap=120))
    alone = run_batch([a])[0]
    mix = run_batch([
        (req_params(64, c2=12.0, so_type=2), dict(seed=3, tol=1e-300, cap=60)),
        a,
        (req_params(128, omeg=0.8), dict(seed=5, tol=1e-300, cap=200, policy=gpspin.POLICY_FP32_REFINE)),
        (req_params(72), dict(seed=7, tol=1e-300, cap=40)),
    ])[1]
    assert alone[0] == mix[0] == gpspin.REQ_DONE
    assert alone[1] == mix[1] == 120
    assert np.array_equal(alone[3], mix[3])
    assert alone[2]["energy"] == mix[2]["energy"]


def test_batched_solve_equals_single_handle():
    p = req_params(80, so_type=2, rabi=0.4)
    st, steps, obs, psi = run_batch([(p, dict(seed=21, tol=1e-300, cap=100))])[0]
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=21, phase_noise=1e-3)
        s.propagate(100, gpspin.IMAG)
        want = s.get_state()
        e = s.observables()["energy"]
    assert np.max(np.abs(psi - want)) <= 1e-13 * np.max(np.abs(want))
    assert abs(obs["energy"] - e) <= 1e-13 * abs(e)


def test_admission_by_footprint_and_retirement():
    p = req_params(64)
    one = gpspin.request_bytes(p)
    with gpspin.Batch(int(2.5 * one), check_every=CHECK) as b:
        ids = [b.submit(p, seed=s, tol=1e-300, cap=40) for s in range(4)]
        nr, nq = b.step()
        assert nr == 2 and nq == 2          # two fit, two wait
        states = [b.poll(i)[0] for i in ids]
        assert states[:2] == [gpspin.REQ_RUNNING] * 2 and states[2:] == [gpspin.REQ_QUEUED] * 2
        nr, nq = b.step()                   # first two reach the cap and retire; the others are admitted
        assert [b.poll(i)[0] for i in ids[:2]] == [gpspin.REQ_DONE] * 2
        assert nr == 2 and nq == 0
        for _ in range(5):
            nr, nq = b.step()
        assert [b.poll(i)[0] for i in ids] == [gpspin.REQ_DONE] * 4
        too_big = b.submit(req_params(256), seed=1, tol=1e-300, cap=20)
        b.step()
        assert b.poll(too_big)[0] == gpspin.REQ_FAILED


def test_convergence_rule_stops_before_the_cap():
    p = req_params(64, c0=80.0, omeg=0.3)
    (st, steps, obs, psi), = run_batch([(p, dict(seed=2, tol=1e-6, cap=20000))])
    assert st == gpspin.REQ_DONE and steps < 20000


def test_mixed_precision_policy_agrees_with_fp64():
    """The FP32-then-FP64 solve agrees with the FP64 solve to |dE/E| <= 1e-6."""
    p = req_params(64, c0=80.0, omeg=0.3)
    r64, r32 = run_batch([
        (p, dict(seed=2, tol=1e-9, cap=6000)),
        (p, dict(seed=2, tol=1e-9, tol32=1e-7, cap=6000, policy=gpspin.POLICY_FP32_REFINE)),
    ])
    assert r64[0] == r32[0] == gpspin.REQ_DONE
    e64, e32 = r64[2]["energy"], r32[2]["energy"]
    assert abs(e32 - e64) <= 1e-6 * abs(e64)


def test_graph_ticks_equal_direct_ticks_bitwise():
    """Ticks replayed from captured CUDA graphs give bitwise the results of ticks
    whose kernels are launched directly, with both precision groups running (on
    their two streams) and the running set changing as solves finish."""
    items = [
        (req_params(64, c2=12.0, so_type=2), dict(seed=3, tol=1e-300, cap=60)),
        (req_params(96), dict(seed=11, tol=1e-300, cap=140)),
        (req_params(128, omeg=0.8), dict(seed=5, tol=1e-300, cap=100, policy=gpspin.POLICY_FP32_REFINE,
                                         refine_steps=40)),
    ]
    a = run_batch(items, graphs=True)
    b = run_batch(items, graphs=False)
    for x, y in zip(a, b):
        assert x[0] == y[0] == gpspin.REQ_DONE and x[1] == y[1]
        assert np.array_equal(x[3], y[3])


def test_persistent_launches_equal_one_cta_per_item_bitwise():
    """Persistent batched launches (CTAs taking the work items from a device
    counter, largest grids first) give bitwise the results of one CTA per work
    item: at one CTA per resident slot, and with the grid capped at a few CTAs
    so that every CTA runs many items and many phases of its staging barrier
    (and the counter is reset between the launches of a tick), with graph and
    direct ticks, both precision groups and a running set that changes."""
    items = [
        (req_params(64, c2=12.0, so_type=2), dict(seed=3, tol=1e-300, cap=60)),
        (req_params(96), dict(seed=11, tol=1e-300, cap=140)),
        (req_params(128, omeg=0.8), dict(seed=5, tol=1e-300, cap=100, policy=gpspin.POLICY_FP32_REFINE,
                                         refine_steps=40)),
        (req_params(80, rabi=0.0), dict(seed=9, tol=1e-300, cap=80, policy=gpspin.POLICY_FP32_REFINE,
                                        refine_steps=20)),
    ]
    ref = run_batch(items, graphs=False, persist=-1)
    for graphs, persist in ((True, 0), (False, 5), (True, 3)):
        got = run_batch(items, graphs=graphs, persist=persist)
        for x, y in zip(ref, got):
            assert x[0] == y[0] == gpspin.REQ_DONE and x[1] == y[1]
            assert np.array_equal(x[3], y[3])


def test_running_limit_admits_by_work_in_flight():
    """With a limit on the grid points of the running solves, requests wait for
    work to finish (arrival order kept, one solve always runs), and their
    results are bitwise those of the unlimited batch."""
    items = [(req_params(64), dict(seed=s, tol=1e-300, cap=40)) for s in range(3)]
    free = run_batch(items)
    out = {}
    with gpspin.Batch(8 << 30, check_every=CHECK) as b:
        b.set_running_limit(64 * 64 + 100)  # room for one 64^2 solve at a time
        ids = [b.submit(p, **kw) for p, kw in items]
        nr, nq = b.step()
        assert (nr, nq) == (1, 2)
        for _ in range(20):
            nr, nq = b.step()
            if nr == 0 and nq == 0:
                break
        for i in ids:
            out[i] = b.poll(i, fetch=True, release=True)
    for f, i in zip(free, ids):
        assert out[i][0] == gpspin.REQ_DONE and np.array_equal(out[i][3], f[3])
