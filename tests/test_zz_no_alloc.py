"""gp_propagate_noalloc: the time step for callers that must not allocate device
memory (their host application owns the GPU memory pool, or they run under a
no-allocation rule), so they cannot create a gp_handle.  The test owns psi in a
torch tensor (the test itself may allocate) and checks the no-allocation entry
point against the handle-based gp_propagate on two calls in a row.

The file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu


def params():
    # ragged 200 x 120 grid with every term of the step switched on
    return dict(nx=200, ny=120, xlen=20.0, ylen=12.0, dt=0.002, c0=90.0, c2=-7.0, omeg=0.6, so_type=1,
                gamma=0.7, rabi=0.3)


@pytest.mark.parametrize("shape", [(200, 120), (256, 256)])
@pytest.mark.parametrize("mode", [gpspin.IMAG, gpspin.REAL])
def test_noalloc_matches_propagate_twice(mode, shape):
    import torch
    gpspin.build()
    p = dict(params(), nx=shape[0], ny=shape[1], xlen=0.1 * shape[0], ylen=0.1 * shape[1])
    psi0 = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=13) \
        + inputs.random_state(p["nx"], p["ny"], seed=14, scale=0.02)
    stream = torch.cuda.Stream()
    dev = torch.from_numpy(psi0.copy()).to("cuda")
    with gpspin.Solver(p) as ref:
        ref.set_state(psi0)
        for call in range(2):
            ref.propagate(15, mode)
            want = ref.get_state()
            torch.cuda.synchronize()
            # after the first call (module loaded, scratch addresses looked up) a
            # call must not take any device memory
            free_before = torch.cuda.mem_get_info()[0]
            gpspin.propagate_noalloc(p, dev.data_ptr(), 15, mode, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            if call == 1:
                assert torch.cuda.mem_get_info()[0] >= free_before
            got = dev.cpu().numpy()
            assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    gpspin.build()
    p = dict(params(), nx=257, ny=16)
    dev = torch.zeros((3, 16, 257), dtype=torch.complex128, device="cuda")
    with pytest.raises(gpspin.GPError) as ei:
        gpspin.propagate_noalloc(p, dev.data_ptr(), 1)
    assert ei.value.status == 6
