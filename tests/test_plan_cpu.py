"""Host-side routing of mps_apply_circuit (mps_plan_image, no GPU needed) against the
Python mirrors that serving and the flop model use, and the largest bond against the
oracle MPS's bond dimensions (Sec. II.B truncation rule)."""
import numpy as np
import pytest

from oracle import circuit as o_circ
from oracle import mps as o_mps
from paper_2607_10280_b300 import flops, synth


@pytest.fixture(scope="module")
def api():
    from paper_2607_10280_b300 import _lib, build
    build.build()
    _lib.lib()
    from paper_2607_10280_b300 import api as a
    return a


def test_routes_match_the_python_mirrors(api):
    for p in range(2, 17):
        for L in range(0, 7):
            for chi in (1, 2, 3, 4, 8, 16, 32, 64, 128, 4096):
                pl = api.plan_image(p, L, chi, "ladder", "mixed")
                assert pl["lossy"] == (flops.lossy(p, L, chi) and L >= 1), (p, L, chi, pl)
                assert (pl["route"] == "operator_product") == (flops.operator_product_path(p, L, chi) and not pl["lossy"]), (p, L, chi, pl)
                if pl["lossy"]:
                    assert pl["route"] == "sequential_complex128"
                    assert api.plan_image(p, L, chi, "ladder", "fp64")["route"] == "sequential"
                    assert api.plan_image(p, L, chi, "ladder", "mixed_fast")["route"] == "sequential"
                if pl["bond"] <= 32:
                    assert pl["padding"] == max(flops.padding(p, chi), 4), (p, L, chi, pl)
                else:
                    assert pl["padding"] >= pl["bond"] or not pl["supported"]
                assert pl["supported"] == (pl["bond"] <= 128)


def test_bonds_match_the_oracle_mps(api):
    for p in (2, 3, 4):
        for L in (1, 2, 3, 5):
            for chi in (1, 2, 3, 4, 8, 64):
                x = synth.uniform_pixels(1, p, seed=5)[0]
                params = synth.circuit_params(L, p * p, seed=6)
                st = o_mps.simulate(o_circ.build_circuit("ladder", x, L, params), p * p, chi)
                pl = api.plan_image(p, L, chi, "ladder", "fp64", layer_pipeline=False)
                assert pl["route"] == "sequential"
                assert pl["bond"] == max(st.bond_dims() + [1]), (p, L, chi, pl, st.bond_dims())
                # generic pixels and angles: a lossy step discards nonzero weight
                assert pl["lossy"] == (float(np.sum(st.discarded)) > 1e-20), (p, L, chi, pl)


def test_plan_rejects_bad_arguments(api):
    from paper_2607_10280_b300._lib import MpsError
    with pytest.raises(MpsError):
        api.plan_image(1, 2, 4)
    with pytest.raises(MpsError):
        api.plan_image(4, -1, 4)
    assert not api.plan_image(5, 8, 4096)["supported"]      # bond 256 above the limit
