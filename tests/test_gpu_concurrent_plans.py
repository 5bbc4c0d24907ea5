"""Two plans searched at once from two host threads.

The plans share the image size but not the array, so their column-FFT and
row-pass kernels ask for different amounts of shared memory.  The kernels'
shared-memory attribute belongs to the kernel, not to the plan, so a plan must
not be able to change it under the other's launches.  Each plan's results
while the other runs must equal its results alone.
"""

import threading

import numpy as np
import pytest

import oracle
import synth
import paper_1802_03084_gb300 as rf
from gpu_common import small_random_segment

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


def _plan(seed, nant, nchan, extent, cell_frac):
    rng = np.random.default_rng(seed)
    seg = small_random_segment(rng, nant, nchan, 48, 256, extent=extent)
    umax = extent * 2.0 * seg["freq_hz"].max() / oracle.C_LIGHT
    plan = rf.Plan(seg["ant_uvw"], seg["freq_hz"], 2e-3, 256, cell_frac / umax, np.linspace(0, 20.0, 3), [1, 2],
                   3.0, flags=rf.RF_EDGE_PARTIAL, max_nint=48)
    plan.set_graphs(False)   # direct launches: every search sets the kernels' attributes again
    return plan, seg


def test_two_plans_of_one_image_size_from_two_threads():
    plans = [_plan(11, 12, 24, 300.0, 0.45), _plan(12, 6, 5, 300.0, 0.12)]
    try:
        info = [p.info() for p, _ in plans]
        assert info[0].iu_max != info[1].iu_max       # different column counts, so different requests
        alone = [p.search_stats(seg["vis"]) for p, seg in plans]
        errors = []
        results = [[], []]

        def run(k):
            p, seg = plans[k]
            try:
                for _ in range(6):
                    results[k].append(p.search_stats(seg["vis"]))
            except Exception as e:  # reported below
                errors.append(e)

        threads = [threading.Thread(target=run, args=(k,)) for k in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for k in range(2):
            c0, s0 = alone[k]
            assert len(results[k]) == 6
            for c, s in results[k]:
                assert np.array_equal(c, c0) and np.array_equal(s, s0)
    finally:
        for p, _ in plans:
            p.close()
