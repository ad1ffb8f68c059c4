"""The allocation-free regularisation entry point (ibl_regularize_noalloc),
called through the C ABI on caller-owned device buffers, gives the same
positions and iteration count as the workspace-based ibl_regularize_now, on
two calls in a row (the second one finds the first one's data left in the
library's fixed scratch array).  It exists for callers that cannot allocate
device memory, e.g. programs whose allocator owns the whole device."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _mesh(level, seed):
    from paper_2403_01161_gb300 import inputs
    from paper_2403_01161_gb300.sim import icosphere

    r, t = icosphere(level, 5.0, (15.5, 15.5, 15.5))
    r = (r - 15.5) * [1.5, 0.8, 0.9] + 15.5
    return inputs.jitter(r, 0.15, seed), t


def test_noalloc_regularize_matches_workspace_path():
    import torch

    from paper_2403_01161_gb300 import _lib as L
    from paper_2403_01161_gb300.sim import Sim

    lib = L.load()
    for level, seed in ((3, 11), (2, 12)):
        r0, t = _mesh(level, seed)
        g = Sim((32, 32, 32), 1.0, np.zeros((1, 3, 3)), 1)
        g.add_mesh(r0, t, 0.01)
        g.set_regularization(0.1, 0.51, 0.01, 100, 0, True)
        it_ref = g.regularize_now()
        r_ref, _, _ = g.mesh()
        ptr, idx = g.neighbours()
        g.close()

        r_dev = torch.tensor(r0, dtype=torch.float64, device="cuda")
        ptr_dev = torch.tensor(ptr, dtype=torch.int32, device="cuda")
        idx_dev = torch.tensor(idx, dtype=torch.int32, device="cuda")
        res = torch.zeros(2, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = lib.ibl_regularize_noalloc(ctypes.c_void_p(r_dev.data_ptr()), ctypes.c_void_p(ptr_dev.data_ptr()),
                                        ctypes.c_void_p(idx_dev.data_ptr()), r0.shape[0], 0.1, 0.51, 0.01, 100, 1,
                                        ctypes.c_void_p(res.data_ptr()), ctypes.c_void_p(stream))
        assert st == L.IBL_OK, lib.ibl_last_error()
        torch.cuda.synchronize()
        assert int(res[0]) == it_ref and int(res[1]) == 1
        assert np.abs(r_dev.cpu().numpy() - r_ref).max() < 1e-12


def test_noalloc_rejects_oversize():
    import torch

    from paper_2403_01161_gb300 import _lib as L

    lib = L.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = lib.ibl_regularize_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                    ctypes.c_void_p(buf.data_ptr()), 16385, 0.1, 0.51, 0.01, 100, 1,
                                    ctypes.c_void_p(buf.data_ptr()), None)
    assert st == L.IBL_EINVAL
    assert b"16384" in lib.ibl_last_error()
