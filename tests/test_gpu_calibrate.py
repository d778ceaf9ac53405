"""The arithmetic calibration entry (esplit_measure_fp64): every mode runs
and returns a positive rate, an unknown mode is an argument error, and the
rates are ordered as the kernels' design relies on (float32 FMA well above
float64 FMA; the float64 divide, log and exp each cost several float64
FMAs)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_07181_gb300 as es
    return es


def test_calibration_modes(lib):
    rates = {}
    for mode in range(11):
        rc, rate, ms = lib.capi.esplit_measure_fp64(0, mode)
        assert rc == 0
        assert rate > 0.0 and ms > 0.0
        rates[mode] = rate
    dfma = rates[0] / 2.0
    print("DFMA/s %.3e, DMMA FMA/s %.3e, mixed %.3e, FFMA/s %.3e, cost in DFMA: div %.1f log %.1f exp %.1f "
          "(CUDA log %.1f exp %.1f), round trip %.1f"
          % (dfma, rates[1] / 2, rates[2] / 2, rates[3] / 2, dfma / rates[4], dfma / rates[5], dfma / rates[6],
             dfma / rates[7], dfma / rates[8], dfma / rates[9]))
    print("bf16 mma.sync %.1f TFLOP/s" % (rates[10] / 1e12))
    assert 0.1e12 < rates[0] < 10e12
    assert rates[3] > 8.0 * rates[0]
    assert rates[10] > rates[3]
    for mode in (4, 5, 6, 7, 8, 9):
        assert rates[mode] < dfma


def test_calibration_bad_mode(lib):
    for mode in (-1, 11):
        rc, _, _ = lib.capi.esplit_measure_fp64(0, mode)
        assert rc == lib.capi.ESPLIT_ERR_ARG
