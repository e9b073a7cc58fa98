"""tc_energy_dev_noalloc: the FP64 energy for callers that cannot allocate device memory.

Such callers (code running inside a runtime that owns every device
allocation, or that must not risk a failing or fragmenting allocation
mid-run) get their scratch from the library's static device array instead of
cudaMalloc.  This file is collected last so that a failure here comes after
every other test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
import paper_2512_01055_gb300 as tc
from paper_2512_01055_gb300 import build

pytestmark = pytest.mark.gpu
RTOL = 1e-9   # the FP64 path's |dE| / |E_T| bound


def _dev(job):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(job, k))).to("cuda")
            for k in ("eps", "t1", "t2", "ovvv", "ovoo", "ovov")}


def _noalloc_call(job, d, e_t, e_ijk):
    """One call through the C ABI (ctypes, no Python wrapper)."""
    import torch
    lib = tc.load()
    ints = tc.tc_ints(d["ovvv"].data_ptr(), d["ovoo"].data_ptr(), d["ovov"].data_ptr())
    buf = ctypes.create_string_buffer(256)
    s = lib.tc_energy_dev_noalloc(job.o, job.v, d["eps"].data_ptr(), d["t1"].data_ptr(), d["t2"].data_ptr(),
                                  ctypes.byref(ints), e_t.data_ptr(), e_ijk.data_ptr(),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), buf, 256)
    assert s == tc.TC_OK, buf.value
    torch.cuda.synchronize()
    return float(e_t.item()), e_ijk.cpu().numpy()


def _scratch_bytes_one_orbit_per_item(o, v, tile=8):
    """Bytes the FP64 path's tables and partial sums need with one tile orbit per work item."""
    al = lambda x: (x + 255) // 256 * 256
    n_trip = o * (o + 1) * (o + 2) // 6 - o
    t = (v + tile - 1) // tile
    n_orb = t * (t + 1) * (t + 2) // 6
    return (al(16 * n_trip) + al(16 * n_orb) + al(16 * n_trip * n_orb) + al(8 * n_trip) + al(32) + al(8))


# (12, 160): one orbit per item would need more than the static array holds,
# so the entry point packs several orbits into each item
@pytest.mark.parametrize("o,v,seed", [(6, 36, synth.WORKLOAD_SEEDS["tiny_o6_v36"]), (5, 29, 3), (12, 160, 7)])
def test_noalloc_matches_context_entry_on_two_calls(o, v, seed):
    import torch
    build.build()
    if (o, v) == (12, 160):
        assert _scratch_bytes_one_orbit_per_item(o, v) > tc.NOALLOC_SCRATCH_BYTES
    job = synth.make_job(o, v, seed)
    d = _dev(job)
    ctx = tc.tc_init(0)
    try:
        ref_ijk = torch.zeros((o,) * 3, dtype=torch.float64, device="cuda")
        ref = tc.tc_energy_dev(ctx, o, v, d["eps"], d["t1"], d["t2"], d["ovvv"], d["ovoo"], d["ovov"],
                               prec=tc.TC_FP64, e_ijk=ref_ijk)
    finally:
        tc.tc_finalize(ctx)
    ref_ijk = ref_ijk.cpu().numpy()
    scale = np.abs(ref_ijk).max()
    e_t = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    e_ijk = torch.full((o,) * 3, np.nan, dtype=torch.float64, device="cuda")
    for call in range(2):                           # the shared array keeps the previous call's contents
        free_before = torch.cuda.mem_get_info()[0]
        e, eijk = _noalloc_call(job, d, e_t, e_ijk)
        if call == 1:                               # after the first call's one-time set-up
            assert torch.cuda.mem_get_info()[0] == free_before
        assert abs(e - ref.e_t) <= RTOL * abs(ref.e_t), (call, e, ref.e_t)
        assert np.all(np.abs(eijk - ref_ijk) <= RTOL * scale), call


def test_noalloc_rejects_jobs_beyond_the_static_array():
    import torch
    build.build()
    lib = tc.load()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    ints = tc.tc_ints(p, p, p)
    buf = ctypes.create_string_buffer(256)
    # v = 4000 -> 500 tiles of 8 -> ~2.1e7 tile orbits: tables alone exceed the array
    s = lib.tc_energy_dev_noalloc(10, 4000, p, p, p, ctypes.byref(ints), p, None, None, buf, 256)
    assert s == tc.TC_ENOMEM
    assert b"too large" in buf.value
    s = lib.tc_energy_dev_noalloc(0, 5, p, p, p, ctypes.byref(ints), p, None, None, buf, 256)
    assert s == tc.TC_EINVAL
