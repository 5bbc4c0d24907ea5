"""The device-side waits are bounded: the row pass's wait on an mbarrier that
nothing arrives at and the fused pass's wait on a count that nothing raises
each give up and report it, and the device stays usable."""

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import compare_stats, plans_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def engine():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_03084_gb300.build import build
    build()
    rf.lib()
    torch.cuda.init()
    yield


def test_wait_gives_up_and_the_context_survives():
    assert rf.rf_selftest_bounded_wait(0, 1000) == 1
    assert rf.rf_selftest_bounded_wait(0, 1) == 1
    with pytest.raises(rf.RfError) as e:
        rf.rf_selftest_bounded_wait(0, 0)
    assert e.value.status == rf.RF_ERR_INVALID_ARG
    # a search right after runs normally
    spec = synth.config("tiny")
    seg = synth.make_segment(spec, nint=40)
    gp, op = plans_for(spec, seg)
    with gp:
        _, gst = gp.search_stats(seg["vis"])
    _, ost = oracle.search_segment(op, seg["vis"], images=[(0, 0, t) for t in range(40)], with_stats=True)
    sub = gst[(gst["dm_idx"] == 0)]
    compare_stats(sub, ost)
