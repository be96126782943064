"""Dense and modal cubes (support_eps = 0): every influence function is
resampled over its whole plane, the case of global modal bases such as the
paper's mirror-mode sets.  Same kernels and the same column criterion as the
zonal parity tests (tests/test_im_parity.py), against the FP64 oracle, which
always uses the dense cube."""
import pytest

from paper_2606_07759_b300 import workloads as W
from test_im_parity import TOL, check_workload

pytestmark = pytest.mark.gpu


def test_dense_scao_small_all_columns():
    assert check_workload(W.dense(W.scao_small())) < TOL


def test_dense_elt_geometry_reduced_all_columns():
    check_workload(W.dense(W.elt_single(seed=2, n_side=21, grid_n=120, n_sub=17)))


def test_modal_cosine_cube_all_columns():
    # 80 global modes (2-D cosines up to order 8) on the SCAO small geometry
    check_workload(W.modal_scao())


def test_dense_mcao_reduced_all_pairs():
    check_workload(W.dense(W.mcao_batched(seed=3, scale=0.2)))


def test_modal_elt_geometry_reduced_all_columns():
    # 200 cosine modes on the reduced ELT pupil (120 px, 17x17 subapertures)
    check_workload(W.modal_elt(n_modes=200, grid_n=120, n_sub=17))


def test_modal_elt_full_scale_sampled_columns():
    # the 4519-mode cube at full ELT scale (480 px, 68x68, M = 544): 24 columns
    check_workload(W.modal_elt(), cols_per_dm=24, seed=5)
