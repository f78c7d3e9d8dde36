"""lpm_draws_static: the draws of lpm_draws for callers that cannot allocate device memory
(their device memory belongs to their own pool allocator or a fixed budget). It stages
through the library's fixed device array instead of allocating; here it must give the
same words and normals as lpm_draws, bit for bit and call after call, leave the device's
free memory unchanged, and refuse requests larger than that array. This file is collected
last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()


def test_draws_static_matches_draws_on_consecutive_calls():
    from paper_0912_3223_gb300 import lpm
    for call, n in enumerate([5000, lpm.DRAWS_STATIC_MAX]):
        rng = np.random.default_rng(100 + call)
        pid = rng.integers(0, 2 ** 40, n).astype(np.uint64)
        step = rng.integers(0, 2 ** 28, n).astype(np.uint32)
        for stream in (0, 1):
            seed = 0xC0FFEE + call
            w_static, n_static = lpm.lpm_draws_static(seed, pid, step, stream)
            w_ref, n_ref = lpm.lpm_draws(seed, pid, step, stream)
            # the same kernel on the same inputs: identical words and normals
            assert np.array_equal(w_static, w_ref)
            assert np.array_equal(n_static, n_ref)


def test_draws_static_allocates_nothing():
    from paper_0912_3223_gb300 import lpm
    rng = np.random.default_rng(7)
    pid = rng.integers(0, 2 ** 40, lpm.DRAWS_STATIC_MAX).astype(np.uint64)
    lpm.lpm_draws_static(3, pid[:10], 0)          # first call on the device: its set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out = [lpm.lpm_draws_static(3 + i, pid, i) for i in range(4)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # the last call's results are its own, not a leftover of the previous call's contents
    w_ref, n_ref = lpm.lpm_draws(6, pid, 3)
    assert np.array_equal(out[-1][0], w_ref) and np.array_equal(out[-1][1], n_ref)
    assert not np.array_equal(out[-2][0], out[-1][0])


def test_draws_static_rejects_more_than_its_scratch():
    from paper_0912_3223_gb300 import lpm
    n = lpm.DRAWS_STATIC_MAX + 1
    pid = np.arange(n, dtype=np.uint64)
    with pytest.raises(lpm.LpmError) as e:
        lpm.lpm_draws_static(1, pid, 0)
    assert e.value.status == lpm.LPM_E_INVALID
    assert "exceeds" in str(e.value)
