"""Host planning of the persistent batch launch (syk_batch_plan, no device needed): how many of
an item's states one CTA takes, and that the launch's shared memory fits the limit."""
import itertools

import pytest

from paper_2002_05725_gb300 import syk

GB300_SMEM = 227 * 1024  # opt-in shared memory per CTA on sm_100-class GPUs


def plan(N, B, m=40, limit=GB300_SMEM):
    return syk.syk_batch_plan(N, B, m, limit)


def test_known_cases_at_the_gb300_limit():
    """The cases the GPU tests run: N <= 24 at 8 states in one CTA, N = 20 at 16, N = 28 at 8
    states as four CTAs of 2, N = 30 one-state items, N = 32 on the per-item path."""
    assert plan(24, 8)[0] == 8
    assert plan(20, 16)[0] == 16
    assert plan(24, 16)[0] == 8     # 2^11 x 16 complex64 = 256 KiB does not fit
    assert plan(28, 8)[0] == 2 and plan(28, 2)[0] == 2
    assert plan(30, 1)[0] == 1
    assert plan(32, 8)[0] == 0 and plan(32, 1)[0] == 0   # 2^15 complex64 = 256 KiB
    assert plan(24, 3)[0] == 0      # only a split into single states would divide 3
    assert plan(24, 12)[0] == 4     # the largest power of two dividing 12
    bs, smem = plan(24, 8)
    assert (1 << 11) * 8 * 8 < smem <= GB300_SMEM


@pytest.mark.parametrize("limit", [48 * 1024, 100 * 1024, GB300_SMEM])
def test_plan_properties(limit):
    for N, B, m in itertools.product(range(4, 34, 2), range(1, 17), (2, 30, 40, 64)):
        bs, smem = plan(N, B, m, limit)
        D = 1 << (N // 2 - 1)
        if bs == 0:
            assert smem == 0
            continue
        assert bs in (1, 2, 4, 8, 16) and B % bs == 0, (N, B, m, bs)
        assert bs > 1 or B == 1, (N, B, m)           # multi-state items split to >= 2 states
        assert D * bs * 8 <= smem <= limit, (N, B, m, bs, smem)   # the staged sector vector fits


def test_plan_monotone_in_limit_and_size():
    """More shared memory never makes a CTA take fewer states, a larger sector never more."""
    for N, B, m in itertools.product(range(8, 34, 2), (1, 2, 4, 8, 16), (30, 40)):
        small, big = plan(N, B, m, 100 * 1024)[0], plan(N, B, m, GB300_SMEM)[0]
        assert small <= big or small == 0, (N, B, m, small, big)
        if N + 2 <= 32:
            assert plan(N + 2, B, m)[0] <= plan(N, B, m)[0] or plan(N, B, m)[0] == 0


def test_plan_rejects_bad_arguments():
    for args in [(5, 8, 40), (2, 8, 40), (24, 0, 40), (24, 8, 1), (24, 8, 65)]:
        with pytest.raises(syk.SykError):
            syk.syk_batch_plan(*args, GB300_SMEM)
