"""The allocation-free column-pointer scan (sic_factor_nnz_noalloc) against the
workspace version (sic_factor_nnz), called through the C-ABI.

sic_factor_nnz_noalloc is for callers that cannot allocate device memory (for instance
code inside a host framework that has reserved the device memory for its own allocator,
or a latency-critical loop that cannot afford cudaMalloc's implicit synchronisation);
its scratch is a static device array inside the library, shared by all calls.  This
file is collected last so that a failure here comes after every other test has run; it
passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import sic
    return torch, sic, sic.Handle(0)


def _counts(torch, n_units, k, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.integers(0, k + 1, n_units).astype(np.int32)).cuda()


@pytest.mark.parametrize("grouped", [False, True])
def test_noalloc_matches_workspace_version_twice(env, grouped):
    torch, sic, h = env
    # two calls in a row with different sizes: the second must not see the first's leftovers
    for n, seed in [(300_001, 1), (5_000, 2)]:
        if grouped:
            rng = np.random.default_rng(seed + 10)
            sizes = rng.integers(1, 65, n)
            sizes = sizes[np.cumsum(sizes) <= n]
            sizes = np.append(sizes, n - sizes.sum()) if sizes.sum() < n else sizes
            gp = np.zeros(len(sizes) + 1, np.int64)
            gp[1:] = np.cumsum(sizes)
            grp = torch.from_numpy(gp).cuda()
            cnt = _counts(torch, len(sizes), 64, seed)
        else:
            grp = None
            cnt = _counts(torch, n, 32, seed)
        ref = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        ws = sic._ws(sic.factor_nnz_workspace(n), "cuda")
        sic.factor_nnz(h, grp, cnt, n, ref, ws)
        out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
        sic.factor_nnz_noalloc(h, grp, cnt, n, out)
        h.sync()
        assert torch.equal(out, ref)
        assert int(out[0]) == 0 and int(out[-1]) > 0


def test_noalloc_rejects_sizes_beyond_scratch(env):
    torch, sic, h = env
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    n_too_big = 65536 * 1024  # n + 1 exceeds the static scratch's 2^26 entries
    code = sic.lib().sic_factor_nnz_noalloc(h.ptr, None, n_too_big, sic._dptr(cnt), n_too_big,
                                            sic._dptr(out), sic._stream(None))
    assert code == sic.SIC_ERR_UNSUPPORTED
