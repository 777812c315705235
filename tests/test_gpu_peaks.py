"""The device throughput probes behind two roofline choices: the FP64 FMA
rate (the FP64 path's denominator) and the cost of one tcgen05 MMA against
N (which set the network convolutions' MMA shape)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1707_08900_gb300 import build
    build.build()


def test_fp64_fma_rate_is_plausible():
    from paper_1707_08900_gb300 import gbfd
    r = gbfd.gbfd_fp64_fma_rate()
    assert 0.2 < r < 10.0


def test_tc_mma_cycles_grow_with_n_and_reach_the_tensor_rate():
    """Cycles per M = 128, K = 16 MMA: never fewer for more columns, twice
    as many for 256 as for 128 columns (the full-rate regime), and the
    full-rate figure within the plausible range of MACs per clock per SM."""
    from paper_1707_08900_gb300 import gbfd
    c = {n: gbfd.gbfd_tc_mma_cycles(n) for n in (16, 32, 48, 64, 96, 128, 256)}
    ns = sorted(c)
    for a, b in zip(ns, ns[1:]):
        assert c[b] >= 0.97 * c[a], c
    assert c[256] == pytest.approx(2 * c[128], rel=0.1), c
    mac_per_clock = 128 * 256 * 16 / c[256]
    assert 1000 < mac_per_clock < 20000, c
    with pytest.raises(gbfd.GbfdError) as e:
        gbfd.gbfd_tc_mma_cycles(40)
    assert e.value.status == 1  # GBFD_ERR_INVALID_ARG
