"""The MCAO dictionary (12 components: 3 DMs and 9 virtual layers up to 22 km
on growing meta-pupils, times 6 LGS sensors = 72 IMs in one launch), reduced
to scale 0.15 so that the FP64 oracle checks every pair, against the same
column criterion as the zonal parity tests."""
import pytest

from paper_2606_07759_b300 import workloads as W
from test_im_parity import check_workload

pytestmark = pytest.mark.gpu


def test_dictionary_reduced_all_pairs():
    wl = W.mcao_dictionary(seed=9, scale=0.15)
    assert len(wl.dms) == 12 and len(wl.wfss) == 6
    check_workload(wl, cols_per_dm=12, seed=3)
