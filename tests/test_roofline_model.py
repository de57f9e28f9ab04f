"""CPU checks of the algorithmic work model behind the roofline numbers: the
FP64 path's face kernel and element kernel together carry exactly the
element pass's algorithmic flops, the FP32 form has no face kernel, and the
per-node counts follow the pair and interface counts of the scheme."""
import pytest

from paper_2607_06045_b300 import roofline as R

W = (5.7, 9.1, 18.1)   # DFMA-equivalents of a reciprocal, square root, logarithm


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_face_and_element_split_keeps_the_total(N):
    K, M = 1000, 50
    nodes = K * (N + 1) ** 2
    work = R.kernel_work(N, 0, K, M, 6 * (N + 1) * M, *W)
    total = R.element_flops(N, 0, *W) * nodes
    assert work["face"][0] + work["element"][0] == pytest.approx(total, rel=1e-12)
    face_row = R.element_ops_per_node(N, 0)["a4_face_flux"]
    assert work["face"][0] == pytest.approx(2.0 * face_row.dfma_eq(*W) * nodes, rel=1e-12)
    # one face-flux evaluation per conforming face: 2 / (N + 1) per node
    assert face_row.inst == pytest.approx(49 * 2.0 / (N + 1))
    assert work["element"][1] == pytest.approx(R.BYTES_PER_NODE_STAGE * nodes)


def test_fp32_form_has_no_face_kernel_and_less_fp64_work():
    work = R.kernel_work(3, 1, 1000, 50, 600, *W)
    assert "face" not in work
    assert R.element_flops(3, 1, *W) < 0.25 * R.element_flops(3, 0, *W)
    # forcing the split on the FP32 form is allowed and still sums up
    w2 = R.kernel_work(3, 1, 1000, 50, 600, *W, face_kernel=True)
    assert w2["face"][0] + w2["element"][0] == pytest.approx(R.element_flops(3, 1, *W) * 16000, rel=1e-12)


def test_pair_fluxes_scale_with_the_degree():
    # N two-point fluxes per node (each pair once), each with one reciprocal
    for N in (2, 4, 6):
        row = R.element_ops_per_node(N, 0)["a2_pair_fluxes"]
        assert row.div == pytest.approx(N)
        assert row.inst == pytest.approx(40 * N)


def test_bytes_per_node_stage():
    # read u^(s), read u^n in two of three stages, write u^(s+1)
    assert R.BYTES_PER_NODE_STAGE == pytest.approx(32 + 64 / 3 + 32)


def test_fp64_time_step_in_two_passes():
    # with the face kernel the time step's FP32 pass reads the state and the
    # faces' wave speeds and carries the method's time-step row (as FP32
    # work); its FP64 pass over the picked elements is not method work
    N, K = 3, 1000
    nodes = K * (N + 1) ** 2
    work = R.kernel_work(N, 0, K, 50, 600, *W)
    assert work["dt_filter"] == (0.0, pytest.approx((32.0 + 8.0) * nodes + 4.0 * K))
    assert work["dt"] == (0.0, pytest.approx(4.0 * K))
    mk = R.method_kernel_work(N, 0, K)
    assert mk["dt"] == (0.0, 0.0)
    assert mk["dt_filter"][0] == 0.0
    assert mk["dt_filter"][1] == pytest.approx(R.method_rows(N)["dt"] * nodes, rel=1e-12)
    # the FP32 form's one-pass time step keeps the row
    assert "dt_filter" not in R.kernel_work(N, 1, K, 50, 600, *W)
    assert "dt_filter" not in R.method_kernel_work(N, 1, K)
