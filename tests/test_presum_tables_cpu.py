"""The pre-summed kernels' staging tables, checked on the host (no GPU): for
every trial of every tile, the library's verifier re-derives from the delay
table where the pass kernel will read and checks the copy lists, the offset
tables and the series' written ranges against it.  Delay tables come from the
oracle (equal to the plan's, which the GPU tests check)."""
import numpy as np
import pytest

import oracle
from paper_1811_04165_gb300 import synth

BEAM_CONFIGS = [(4, 16, 8, 1, 16, 2), (4, 16, 8, 1, 16, 1), (8, 8, 4, 2, 16, 2), (4, 8, 4, 2, 12, 2),
                (2, 32, 2, 1, 8, 1)]


@pytest.mark.parametrize("cfg", BEAM_CONFIGS)
def test_beam_tables_verify(lib, cfg):
    wl = synth.apertif_beam()
    d = oracle.delay_table(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, wl.dms)
    lib.sps_presum_tables_verify(d, wl.channels, wl.n_t, lib.DedispConfig(*cfg))


@pytest.mark.parametrize("C", [37, 38, 39, 40, 61])
@pytest.mark.parametrize("cfg", [(1, 4, 1, 1, 2, 2), (4, 8, 2, 2, 12, 2), (4, 8, 2, 2, 12, 1), (8, 4, 2, 4, 8, 2)])
def test_ragged_tables_verify(lib, C, cfg):
    dms = synth.dm_grid(29, 0.31)
    d = oracle.delay_table(1300.0, 1500.0, C, 65.536e-6, dms)
    lib.sps_presum_tables_verify(d, C, 1003, lib.DedispConfig(*cfg))


@pytest.mark.parametrize("presum", [1, 2])
def test_subband_step_one_tables_verify(lib, presum):
    wl = synth.apertif_beam(subband=True)
    d1, d2 = oracle.subband_tables(wl.f_lo, wl.f_hi, wl.channels, wl.t_samp, 32, wl.coarse_dms, wl.dms)
    n_1, _ = oracle.subband_lengths(wl.n_t, d1, d2)
    cfg = lib.DedispConfig(1, 16, 8, 1, 8, 2) if presum == 2 else lib.DedispConfig(4, 16, 8, 1, 16, 1)
    lib.sps_presum_tables_verify(d1, wl.channels // 32, n_1, cfg)


def test_verifier_flags_reads_beyond_the_written_range(lib):
    """A planted mistake: series written for one output fewer than are read."""
    dms = synth.dm_grid(29, 0.31)
    d = oracle.delay_table(1300.0, 1500.0, 40, 65.536e-6, dms)
    cfg = lib.DedispConfig(4, 8, 2, 2, 12, 2)
    lib.sps_presum_tables_verify(d, 40, 1003, cfg)
    with pytest.raises(lib.SpsError) as e:
        lib.sps_presum_tables_verify(d, 40, 1003 - 8, cfg, read_n_out=1003)
    assert "written range" in str(e.value)
