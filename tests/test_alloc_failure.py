"""Out-of-memory paths of the create calls.

With SMRE_TEST_FAIL_ALLOC=N the N-th device or pinned host allocation of one
create call fails as if memory had run out (include/smre.h).  For every create
call of the C ABI -- a single-image handle (register-band persistent plan, and
the one-image batch a 16-bit handle uses), a batch, a request server, the ADMM
estimator -- each allocation in turn is made to fail: the call must return
SMRE_ENOMEM and leave the device's free memory as it found it; once N passes
the last allocation the call succeeds.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


SIDES = [1, 2, 3, 4]


def _cases(smre):
    cS = smre.smre_bounds(smre.make_params(64, 64, SIDES))
    kw = dict(cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS)
    return {
        "projector": lambda: smre.Projector(96, 128, SIDES, max_cycles=4, **kw),
        "projector_bf16": lambda: smre.Projector(96, 128, SIDES, max_cycles=4, q_dtype=1, **kw),
        "batch": lambda: smre.Batch(SIDES, max_cycles=4, max_images=3, device_bytes=32 << 20, **kw),
        "server": lambda: smre.Server(SIDES, max_cycles=4, max_images=3, device_bytes=32 << 20, **kw),
        "admm": lambda: smre.Admm(64, 64, SIDES, 1.0, max_cycles=4, max_iters=2, **kw),
    }


@pytest.mark.parametrize("name", ["projector", "projector_bf16", "batch", "server", "admm"])
def test_every_allocation_failure_returns_enomem_and_frees_all(torch_cuda, name):
    import paper_1503_03492_gb300 as smre

    make = _cases(smre)[name]
    make().close()                           # first use: the runtime's own set-up
    torch_cuda.cuda.synchronize()
    n = 0
    try:
        while True:
            os.environ["SMRE_TEST_FAIL_ALLOC"] = str(n)
            torch_cuda.cuda.synchronize()
            free0 = torch_cuda.cuda.mem_get_info()[0]
            try:
                obj = make()
            except smre.SmreError as e:
                assert e.status == smre.SMRE_ENOMEM, (n, e.status, str(e))
                torch_cuda.cuda.synchronize()
                assert torch_cuda.cuda.mem_get_info()[0] == free0, (name, n)
                n += 1
                assert n < 200
                continue
            obj.close()
            break
    finally:
        os.environ.pop("SMRE_TEST_FAIL_ALLOC", None)
    assert n >= 3, n                          # several allocations were exercised
    # unset, the hook has no effect
    obj = make()
    obj.close()
