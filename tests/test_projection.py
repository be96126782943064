"""Tomographic projection on the GPU (synim_projection_matrix / _opt)
against the FP64 oracle (oracle/projection.py), on the 12-component MCAO
dictionary reduced to scale 0.15 (80 px pupil grid, 3 directions).

Criteria:
  - projection matrices: max |P_gpu - P_ref| <= 1e-5 x max |P_ref| (FP32
    coordinates and bilinear resample against FP64, as the IM columns);
  - P_opt at lambda = 1e-2 x mean diag(P_DM^T P_DM) (condition number ~2e3):
    max |P_opt_gpu - P_opt_ref| <= 1e-3 x max |P_opt_ref|.  The normal
    matrices come from box-sparse products (each column is non-zero only on
    its actuator's footprint box per direction) and the system is factored
    in FP32, so the solution carries ~cond x 1e-7 relative error;
  - the projection of a component onto itself at a vanishing lambda is the
    identity;
  - lambda = 0 with a component that no direction sees (zero columns) is
    reported as SYNIM_ERR_NOT_CONVERGED.
"""
import numpy as np
import pytest

from oracle import projection as PR
from paper_2606_07759_b300 import abi
from paper_2606_07759_b300 import workloads as W

pytestmark = pytest.mark.gpu

DIRS = [(0.0, 0.0), (8e-5, 0.0), (0.0, -8e-5)]
DMS, LAYERS = [0, 1, 2], list(range(3, 12))


@pytest.fixture(scope="module")
def setup():
    from paper_2606_07759_b300.synim import SynIM
    wl = W.mcao_dictionary(seed=9, scale=0.15)
    s = SynIM(wl.dms, wl.wfss)
    yield wl, s
    s.close()


@pytest.mark.parametrize("b", [1, 2, 4])
def test_projection_matrix_matches_oracle(setup, b):
    wl, s = setup
    comps = [0, 4, 11]
    ref = PR.stack(wl, comps, 0, DIRS, b)
    gpu = s.projection_matrix(0, DIRS, b, comps).cpu().numpy().T
    assert gpu.shape == ref.shape
    err = np.abs(gpu - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err


def test_popt_matches_oracle(setup):
    wl, s = setup
    Pd, Pl = PR.stack(wl, DMS, 0, DIRS, 2), PR.stack(wl, LAYERS, 0, DIRS, 2)
    lam = 1e-2 * np.mean(np.diag(Pd.T @ Pd))
    ref = PR.p_opt(Pd, Pl, lam)
    gpu = s.projection_opt(0, DIRS, 2, DMS, LAYERS, lam).cpu().numpy()
    assert gpu.shape == ref.shape
    err = np.abs(gpu - ref).max() / np.abs(ref).max()
    assert err <= 1e-3, err


def test_popt_of_a_component_onto_itself_is_identity(setup):
    wl, s = setup
    P = PR.stack(wl, [0], 0, DIRS, 2)
    lam = 1e-9 * np.mean(np.diag(P.T @ P))
    X = s.projection_opt(0, DIRS, 2, [0], [0], lam).cpu().numpy()
    np.testing.assert_allclose(X, np.eye(X.shape[0]), atol=2e-3)


def test_singular_normal_matrix_is_reported(setup):
    wl, s = setup
    # seen from 0.01 rad off axis the 22 km layer's footprint moves by 220 m,
    # off its grid: every column is zero and P^T P + 0 I is singular
    far = [(0.01, 0.0)]
    P = PR.stack(wl, [11], 0, far, 2)
    assert not P.any()
    with pytest.raises(abi.SynimError) as ex:
        s.projection_opt(0, far, 2, [11], [0], 0.0)
    assert ex.value.status == 6   # SYNIM_ERR_NOT_CONVERGED
