"""The flop convention of Sec. VI.A reproduces Table 2's printed Tflops."""
import os

import pytest

from paper_1412_0659_gb300 import FLOPS_PC, FLOPS_PP, tree_force_flops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_flops.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append((f[0], *map(float, f[1:])))
    return rows


def test_per_interaction_counts():
    assert (FLOPS_PP, FLOPS_PC) == (23, 65)


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r[0])
def test_table2_gpu_and_application_tflops(row):
    _, ngpu, npg, pp, pc, t_grav, t_tot, gpu_tf, app_tf = row
    n = ngpu * npg
    flops = tree_force_flops(n * pp, n * pc)
    # printed to 3 significant figures (GPU) and 3-5 (application)
    assert flops / t_grav / 1e12 == pytest.approx(gpu_tf, rel=0.005)
    assert flops / t_tot / 1e12 == pytest.approx(app_tf, rel=0.02)
