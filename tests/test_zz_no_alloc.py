"""The no-allocation de-dispersion entry point against the allocating one.

sps_dedisperse_noalloc is for callers that cannot allocate device memory when
they run (a real-time beam loop held to a fixed device-memory footprint once
observing, or code handed only its input and output buffers).  It must return
exactly what sps_dedisperse returns with a caller-provided workspace, call
after call, although every call reuses the same static scratch.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_1811_04165_gb300 import synth

pytestmark = pytest.mark.gpu


def _workload(which):
    if which == "tiny":
        return synth.tiny_brute()
    if which == "subband-small":
        dms = synth.dm_grid(48, 1.3)
        return synth.Workload("subband-small", 96, 1250.0, 1550.0, 81.92e-6, 3001, dms,
                              np.array([1, 4, 16], np.int32), seed=31, n_subbands=8, coarse_dms=dms[::8].copy(),
                              pulses=[synth.Pulse(30.0, 4.0, 40.0, 900.0)])
    return synth.apertif_beam()


@pytest.mark.parametrize("which", ["tiny", "subband-small", "apertif"])
def test_noalloc_matches_the_workspace_entry_point_twice(lib, which):
    import torch
    wl = _workload(which)
    p = lib.Plan.from_workload(wl)
    if which == "apertif":  # the single-channel kernel's staging fits the static scratch
        c = p.config
        c.brute.presum = 0
        p.config = c
    x = synth.filterbank(wl.channels, wl.f_lo, wl.f_hi, wl.t_samp, p.input_samples, wl.seed, wl.pulses,
                         pitch=p.pitch)
    xd = torch.from_numpy(x).cuda()
    shape = (wl.dms.size, wl.n_t)
    want = torch.empty(shape, dtype=torch.int32, device="cuda")
    lib.sps_dedisperse(p, xd, want, workspace=p.workspace())
    for _ in range(2):  # the second call finds the first call's contents in the scratch
        got = torch.full(shape, -1, dtype=torch.int32, device="cuda")
        lib.sps_dedisperse_noalloc(p, xd, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want)  # integer sums: exact
    assert p.status() == 0


def test_noalloc_rejects_plans_beyond_its_scratch(lib):
    import torch
    wl = synth.apertif_beam(subband=True)  # shifted copies plus step-one series: about 148 MB
    p = lib.Plan.from_workload(wl)
    xd = torch.zeros((wl.channels, p.pitch), dtype=torch.uint8, device="cuda")
    D = torch.empty((wl.dms.size, wl.n_t), dtype=torch.int32, device="cuda")
    with pytest.raises(lib.SpsError) as e:
        lib.sps_dedisperse_noalloc(p, xd, D)
    assert e.value.status == 2 and "static scratch" in str(e.value)
