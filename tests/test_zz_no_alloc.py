"""mpm_sort_keys_static: the stable key sort for callers that cannot allocate
device memory (a program whose allocator already holds the GPU's free memory,
or a loop that must not allocate once running).  Its scratch is a fixed
array inside the library, so it allocates nothing.

Checked through the C-ABI against the allocating mpm_sort_keys on the same
keys, on two calls in a row (the second reuses the array the first left
behind), plus the size limit.  This file is collected last so that a run that
stops at the first failure has already run every other test; it passes both
alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - runs only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1909_13380_gb300 import mpm  # noqa: E402


def _keys(n, bits, seed):
    rng = np.random.default_rng(seed)
    hi = (1 << bits) if bits < 32 else (1 << 32)
    return rng.integers(0, hi, size=n, dtype=np.uint64).astype(np.uint32)


def test_static_sort_matches_the_allocating_sort_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    cases = [(300_001, 20, 1), (mpm.MPM_SORT_STATIC_MAX_KEYS, 32, 2)]
    for n, bits, seed in cases:
        keys = _keys(n, bits, seed)
        dk = torch.from_numpy(keys.view(np.int32)).cuda()
        ref = torch.empty(n, dtype=torch.int32, device="cuda")
        got = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        mpm.mpm_sort_keys(dk, ref, n, bits)
        mpm.mpm_sort_keys_static(dk, got, n, bits)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.array_equal(g, r)
        assert np.array_equal(r, np.argsort(keys, kind="stable").astype(np.int32))


def test_static_sort_rejects_more_keys_than_its_scratch_holds():
    n = mpm.MPM_SORT_STATIC_MAX_KEYS + 1
    dk = torch.zeros(n, dtype=torch.int32, device="cuda")
    dp = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(mpm.MPMError) as ei:
        mpm.mpm_sort_keys_static(dk, dp, n, 8)
    assert ei.value.status == mpm.MPM_ERR_ARG


def test_static_sort_allocates_no_device_memory():
    # the reason the entry point exists: once the library is loaded, a call
    # leaves the device's free memory exactly as it found it
    n, bits = 500_000, 24
    keys = _keys(n, bits, 5)
    dk = torch.from_numpy(keys.view(np.int32)).cuda()
    got = torch.empty(n, dtype=torch.int32, device="cuda")
    mpm.mpm_sort_keys_static(dk, got, n, bits)      # first call: loads the device code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    mpm.mpm_sort_keys_static(dk, got, n, bits)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(got.cpu().numpy(), np.argsort(keys, kind="stable").astype(np.int32))
