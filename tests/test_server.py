"""Continuous-batching request loop (smre_server_*).

Requests of different sizes arrive from several threads while others are on
the GPU; each result must equal, bit for bit, the same image projected alone
(with FP32 and with BF16 increments), and the latency counters must account
for every request.
"""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smre():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_1503_03492_gb300 as m
    return m


@pytest.mark.parametrize("q_dtype", [0, 1])      # FP32 and BF16 increments
def test_served_results_equal_alone_and_counters(smre, oracle_mod, q_dtype):
    from synthetic import sofi_like
    sides = list(range(1, 6))
    cS = oracle_mod.bounds(sides, 0.9)
    kw = dict(cmode=smre.SMRE_C_EXPLICIT, c_explicit=list(cS), max_cycles=80, tol=1e-5,
              tol_relative=True, q_dtype=q_dtype)
    sizes = [64, 96, 130, 64, 200, 77, 128, 256, 90, 64, 150, 100]
    imgs = [np.ascontiguousarray(sofi_like(side=s, frames=40, seed=500 + i), np.float32)
            for i, s in enumerate(sizes)]
    # each image alone
    alone = []
    for x in imgs:
        out = np.full_like(x, np.nan)
        with smre.Batch(sides, max_images=1, device_bytes=64 << 20, **kw) as B:
            (r,) = B.project([x], [out])
        alone.append((out, r.cycles))
    # served: a small arena forces queueing; three submitting threads
    outs = [np.full_like(x, np.nan) for x in imgs]
    tickets = [None] * len(imgs)
    with smre.Server(sides, cycles_per_round=3, max_images=4, device_bytes=48 << 20, **kw) as S:
        def client(k):
            for i in range(k, len(imgs), 3):
                tickets[i] = S.submit(imgs[i], outs[i])
                time.sleep(0.002 * (i % 4))
        th = [threading.Thread(target=client, args=(k,)) for k in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        res = [S.wait(t) for t in tickets]
        st = S.stats()
    assert st.submitted == st.completed == len(imgs)
    assert 1 <= st.peak_active <= 4 and st.waiting == 0 and st.active == 0
    assert 0 < st.p50_s <= st.p99_s <= st.max_s and st.images_per_s > 0
    for (a, cyc), o, r in zip(alone, outs, res):
        assert r.cycles == cyc
        assert np.array_equal(a, o)


def test_server_rejects_what_can_never_fit(smre):
    with smre.Server([1, 2, 4], max_images=2, device_bytes=4 << 20, max_cycles=5) as S:
        big = np.zeros((512, 512), np.float32)
        with pytest.raises(smre.SmreError):
            S.submit(big, np.empty_like(big))            # needs more than the whole arena
        with pytest.raises(smre.SmreError):
            S.submit(np.zeros((8, 3000), np.float32), np.empty((8, 3000), np.float32))
        x = np.ones((32, 32), np.float32) * 3.0
        out = np.empty_like(x)
        t = S.submit(x, out)
        r = S.wait(t, timeout_s=30.0)
        assert r is not None and r.cycles == 5
        assert np.isfinite(out).all()
