"""The benchmark's roofline accounting (host only): the method's minimum bytes
per stage are 16 B per field-DOF plus 64 B per element in FP32, i.e. 16.40 B
per field-DOF at N = 3 and 16.21 B at N = 4 on the layered workload; the
kernel's own minimum adds its mesh tables and stored factor on top."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("N,per_dof", [(3, 16.40), (4, 16.21)])
def test_method_minimum_bytes_per_dof(N, per_dof):
    K = 524288
    nodes = K * (N + 1) ** 2 * (N + 2) // 2
    a = bench._alg_bytes_per_stage(K, nodes)
    assert a / (4 * nodes) == pytest.approx(per_dof, abs=0.005)
    kb = bench._kernel_bytes_per_stage(K, 282897, nodes, N=N, mass="stored")
    nt = (N + 1) * (N + 2) // 2
    assert kb - a == K * (100 + 4 * nt * (nt + 1) // 2 - 64)


def test_flop_count_is_of_the_expected_size():
    # about 94-105 flop per field-DOF at N = 3 and 133-150 at N = 4 (in-stage factor):
    # D_t, M^tri on four vectors, two triangular sweeps, D_r/D_s, faces and update
    f3 = bench._flops_per_wedge(3, "onthefly") / (4 * 40)
    f4 = bench._flops_per_wedge(4, "onthefly") / (4 * 75)
    assert 90 < f3 < 120 and 125 < f4 < 170
    assert bench._flops_per_wedge(3, "stored") < bench._flops_per_wedge(3, "onthefly")
