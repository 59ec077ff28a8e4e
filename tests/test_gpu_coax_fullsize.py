"""Sec. III.B at full size: the co-axial (10,10)/(20,20) capacitor 100 cells long (12,000 sites, 1D boundary term).

The oracle cannot assemble 12,000 sites, so the full size is checked through properties that hold at any size:
C0/L of the 100-cell tube equals that of the 10-cell tube (a per-length quantity of a periodic system) to 1e-8,
the 10-cell value matches the oracle, and C0/L lies a few per cent above 2 pi eps0 / ln(R2/R1).  The 100-cell
capacitance uses the FP32 factor with FP64 refinement (no 12,000^2 inverse)."""
import math

import numpy as np
import pytest

from gpu_util import make_ctx, need_gpu
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu

ALPHA, RCUT = 0.15, 24.0


def _tube(cells):
    return s.coaxial_tubes(cells, alpha=ALPHA, rcut=RCUT, ktol=1e-8)


def test_coaxial_capacitor_100_cells():
    need_gpu()
    el10 = _tube(10)
    c10 = make_ctx(el10).setup(el10)
    C10 = c10.cpm_capacitance()[1, 1] / el10.box[2]
    C10_ir = c10.cpm_capacitance_ir()[0][1, 1] / el10.box[2]
    ref = o.electrode_capacitance(o.capacitance_matrix(o.assemble_A(el10)), el10)[1, 1] / el10.box[2]
    assert abs(C10 / ref - 1) <= 1e-9 and abs(C10_ir / ref - 1) <= 1e-9
    el100 = _tube(100)
    assert el100.n == 12000
    c100 = make_ctx(el100)
    import torch
    from gpu_util import dev
    c100.cpm_assemble(dev(el100.xyz), dev(el100.eta), dev(el100.group, torch.int32), el100.n_groups)
    C, it, res = c100.cpm_capacitance_ir()
    C100 = C[1, 1] / el100.box[2]
    assert res < 1e-12
    assert abs(C100 / C10 - 1) <= 1e-8
    ana = 2 * math.pi * o.EPS0 / math.log(s.tube_radius(20) / s.tube_radius(10))
    assert 0 < C100 / ana - 1 < 0.1
