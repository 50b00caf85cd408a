"""Host checks of the seeded workload generators (no GPU)."""
import numpy as np
import pytest

from workloads import stack_config
from workloads.thiim_workloads import LayeredStack


@pytest.mark.parametrize("st", [stack_config("stack32"), stack_config("adjoint128"),
                                LayeredStack(nx=40, ny=20, nz=48, seed=3),
                                LayeredStack(nx=16, ny=16, nz=32, eps_scale=1.3)])
def test_material_map_reproduces_the_permittivity(st):
    ids = st.material_ids()
    assert ids.dtype == np.uint8 and ids.shape == (st.nz, st.ny, st.nx)
    assert np.array_equal(st.material_eps()[ids], st.eps())
    # every layer of the stack is present
    assert set(np.unique(ids)) == {0, 1, 2, 3}


def test_material_map_planes_match_the_whole_map():
    st = stack_config("stack32")
    assert np.array_equal(st.material_id_planes(10, 20), st.material_ids()[10:20])
