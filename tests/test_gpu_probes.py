"""Probes beside the walk path: the device Philox4x32-10 against the
oracle's, bit for bit on 10^6 counters (with counter word 0 wrapping), and the
random-gather and Philox rate probes return sane figures."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1903_11749_gb300 import build as B
    B.build()
    from paper_1903_11749_gb300 import ppr
    return ppr.Context(0)


@pytest.mark.parametrize("seed,counter", [(1, (0, 0, 0, 0)), (0xDEADBEEF12345678, (2**32 - 500_000, 7, 123456, 9)),
                                          (2**64 - 1, (17, 2**32 - 1, 2**31, 2**32 - 1))])
def test_device_philox_equals_oracle(ctx, oracle, seed, counter):
    n = 1_000_000
    got = ctx.probe_philox(seed, counter, n)
    want = oracle.philox4x32_run(counter, [seed & 0xFFFFFFFF, seed >> 32], n)
    assert np.array_equal(got, want)


def test_rate_probes(ctx):
    from paper_1903_11749_gb300 import ppr
    gather, ms = ctx.probe_rate(0, 2 << 30)  # 2 GiB, far above L2
    assert ms > 0 and 1e9 < gather * 32 < 2e13  # bytes/s between 1 GB/s and 20 TB/s
    indep, ms = ctx.probe_rate(2, 2 << 30)
    assert ms > 0 and 1e9 < indep * 32 < 2e13
    draws, ms = ctx.probe_rate(1)
    assert ms > 0 and draws > 1e10
    with pytest.raises(ppr.PPRError):
        ctx.probe_rate(3)
    with pytest.raises(ppr.PPRError):
        ctx.probe_rate(0, 1000)
