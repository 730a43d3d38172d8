"""The allocation-free energy entry point against the allocating one, through the C-ABI.

pt_energy_fp64_noalloc serves callers that cannot let this library allocate GPU memory
(a host application whose own pool owns the device memory, a loop that cannot take an
allocation's implicit synchronisation, a plug-in where only the host allocates). It keeps
its partial sums in a fixed device array instead of per-context scratch. This file is
collected last so that a failure here does not hide any other test's result.
"""
import numpy as np
import pytest

import oracle
from paper_1107_3490_gb300 import inputs, pt

pytestmark = pytest.mark.gpu


def _reference(x, lj_bonded):
    h = pt.pt_create(10, 1, np.array([1.0]), 1)
    try:
        return pt.pt_energy_fp64(h, x, lj_bonded)
    finally:
        pt.pt_destroy(h)


@pytest.mark.parametrize("N,n_conf,lj_bonded", [(2, 3, 1), (37, 5, 1), (300, 4, 0), (1000, 3, 1)])
def test_noalloc_matches_allocating_entry_point_twice(N, n_conf, lj_bonded):
    import torch
    from paper_1107_3490_gb300 import build
    build.build()
    x = inputs.random_coil(N, n_conf, 7 + N)
    ref = _reference(x, lj_bonded)
    conf = torch.from_numpy(x).cuda()            # the caller's device buffers
    stream = torch.cuda.current_stream().cuda_stream
    orc = np.array([oracle.full_energy(x[c], lj_bonded) for c in range(n_conf)])  # Eq. 4 in FP64
    outs = [torch.full((n_conf,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free_before = None
    for k in range(2):                            # two calls in a row share the array
        pt.pt_energy_fp64_noalloc(conf.data_ptr(), N, n_conf, lj_bonded, outs[k].data_ptr(), stream)
        torch.cuda.synchronize()
        if k == 0:
            free_before = torch.cuda.mem_get_info()[0]
        np.testing.assert_allclose(outs[k].cpu().numpy(), ref, rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(outs[k].cpu().numpy(), orc, rtol=1e-11, atol=1e-10)
    # the call after the first (which looked up the array's address) takes no device memory
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_oversized_and_host_buffers():
    import torch
    N = 1000  # 64 chunks per conformation
    too_many = pt.PT_NOALLOC_SCRATCH_DOUBLES // 64 + 1
    conf = torch.zeros((2, N, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = pt.lib().pt_energy_fp64_noalloc(conf.data_ptr(), N, too_many, 1, out.data_ptr(), None)
    assert rc == pt.PT_EINVAL and "scratch" in pt.pt_last_error()
    host = np.zeros((2, 10, 3), dtype=np.float32)
    rc = pt.lib().pt_energy_fp64_noalloc(host.ctypes.data, 10, 2, 1, out.data_ptr(), None)
    assert rc == pt.PT_EINVAL
