"""The contact sums' capacity (per vertex and contact pass) is checked, not assumed.

Each vertex's contact corrections are summed as packed 32-bit fixed-point
fields with every contribution clamped, so up to 2047 contributions per vertex
and pass are exact; more could wrap a field, and the step reports
VIPER_ECONTACTS instead of a wrong result.  A star of N two-vertex rods crossing
at one point gives every vertex N - 1 interpenetrating neighbours in the first
contact pass: N = 2100 must report the error, N = 1000 must not.
"""
import numpy as np
import pytest

from paper_1906_05260_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _star(n_rods, seed=5, length=0.01, radius=0.001):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_rods, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pos = np.zeros((2 * n_rods, 3))
    pos[0::2] = -0.5 * length * d
    pos[1::2] = 0.5 * length * d
    off = np.arange(n_rods + 1, dtype=np.int32) * 2
    return S.Scene(
        name="star", rod_offsets=off, rest_pos=pos, rest_quat=S.quat_from_z(d), radius=np.full(2 * n_rods, radius),
        density=np.full(n_rods, 1000.0), c_stretch=np.full(n_rods, 1e-7), c_bend=np.full(n_rods, 1e-7),
        c_volume=np.full(n_rods, 1e-7), group=np.arange(n_rods, dtype=np.int32), gravity=np.zeros(3),
        pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)),
        bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=True, volume=True,
        dt=1.0 / 60.0, substeps=1, iterations=1, frames=1)


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1906_05260_gb300 import viper as V
    return V


@pytest.mark.parametrize("solver", ["batched", "plain"])
def test_too_many_contacts_on_one_vertex_are_reported(V, solver):
    sc = _star(2100)
    mode = V.SOLVER_BATCHED if solver == "batched" else V.SOLVER_PLAIN
    g = V.Scene(sc, max_pairs=2100 * 2100 // 2 + 1024, solver=mode)
    g.step(check=False)
    assert g.sync() == V.ECONTACTS
    assert V.error_string(V.ECONTACTS).startswith("over 2047 contact corrections")
    g.close()


@pytest.mark.parametrize("solver", ["batched", "plain"])
def test_many_contacts_below_the_limit_are_summed(V, solver):
    n = 1000
    sc = _star(n)
    mode = V.SOLVER_BATCHED if solver == "batched" else V.SOLVER_PLAIN
    g = V.Scene(sc, max_pairs=n * n // 2 + 1024, solver=mode)
    g.step(check=False)
    assert g.sync() == 0
    assert g.pairs().shape[0] == n * (n - 1) // 2  # every pair of the star touches
    x = g.get_state()["x4"]
    assert np.isfinite(x).all()
    g.close()
