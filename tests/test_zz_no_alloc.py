"""The allocation-free column-pointer scan (sic_factor_nnz_noalloc) against the
workspace version (sic_factor_nnz), called through the C-ABI, and against the plain
definition of col_ptr (an exclusive prefix sum of the per-column entry counts, computed
here with numpy).

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

MAX_LEN = 65536 * 1024  # n + 1 entries the static scratch can scan (2^26)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import sic
    return torch, sic, sic.Handle(0)


def _problem(n, grouped, seed):
    """Host counts (and group offsets) of a random pattern over n columns."""
    rng = np.random.default_rng(seed)
    if not grouped:
        return None, rng.integers(0, 33, n).astype(np.int32)
    sizes = rng.integers(1, 65, n // 16 + 64)
    sizes = sizes[np.cumsum(sizes) <= n]
    if sizes.sum() < n:
        sizes = np.append(sizes, n - sizes.sum())
    gp = np.zeros(len(sizes) + 1, np.int64)
    gp[1:] = np.cumsum(sizes)
    return gp, rng.integers(0, 65, len(sizes)).astype(np.int32)


def _expected(n, gp, cnt):
    """col_ptr by definition: column i of a single-column pattern holds 1 + cnt[i] entries;
    member a of a group of m holds (m - a) + cnt[g]; col_ptr is their exclusive prefix sum."""
    if gp is None:
        per = 1 + cnt.astype(np.int64)
    else:
        m = np.diff(gp)
        g_of = np.repeat(np.arange(len(m)), m)
        a = np.arange(n) - gp[g_of]
        per = (m[g_of] - a) + cnt[g_of].astype(np.int64)
    out = np.zeros(n + 1, np.int64)
    np.cumsum(per, out=out[1:])
    return out


def _both(torch, sic, h, n, gp, cnt, stream=None):
    grp = torch.from_numpy(gp).cuda() if gp is not None else None
    c = torch.from_numpy(cnt).cuda()
    ref = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    ws = sic._ws(sic.factor_nnz_workspace(n), "cuda")
    sic.factor_nnz(h, grp, c, n, ref, ws, stream=stream)
    out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
    sic.factor_nnz_noalloc(h, grp, c, n, out, stream=stream)
    return grp, c, ref, out


@pytest.mark.parametrize("grouped", [False, True])
def test_noalloc_matches_workspace_version_twice(env, grouped):
    torch, sic, h = env
    # two calls in a row with different sizes: the second must not see the first's leftovers
    for n, seed in [(300_001, 1), (5_000, 2)]:
        gp, cnt = _problem(n, grouped, seed)
        _, _, ref, out = _both(torch, sic, h, n, gp, cnt)
        h.sync()
        assert torch.equal(out, ref)
        assert np.array_equal(out.cpu().numpy(), _expected(n, gp, cnt))


def test_noalloc_largest_accepted_size(env):
    """n + 1 = 2^26: the scan uses every tile slot of the static scratch, and the total lands
    in its last entry."""
    torch, sic, h = env
    n = MAX_LEN - 1
    gp, cnt = _problem(n, True, 3)
    grp, c, ref, out = _both(torch, sic, h, n, gp, cnt)
    h.sync()
    assert torch.equal(out, ref)
    assert np.array_equal(out.cpu().numpy(), _expected(n, gp, cnt))
    del grp, c, ref, out
    torch.cuda.empty_cache()


def test_noalloc_two_streams_ordered_by_an_event(env):
    """Calls on two streams share the scratch; ordered by an event (the serialisation the
    header asks for) both results are exact."""
    torch, sic, h = env
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    n1, n2 = 200_003, 70_001
    gp1, cnt1 = _problem(n1, True, 4)
    gp2, cnt2 = _problem(n2, False, 5)
    g1 = torch.from_numpy(gp1).cuda()
    c1 = torch.from_numpy(cnt1).cuda()
    c2 = torch.from_numpy(cnt2).cuda()
    o1 = torch.full((n1 + 1,), -7, dtype=torch.int64, device="cuda")
    o2 = torch.full((n2 + 1,), -7, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    sic.factor_nnz_noalloc(h, g1, c1, n1, o1, stream=s1)
    ev = torch.cuda.Event()
    ev.record(s1)
    s2.wait_event(ev)
    sic.factor_nnz_noalloc(h, None, c2, n2, o2, stream=s2)
    torch.cuda.synchronize()
    h.sync()
    assert np.array_equal(o1.cpu().numpy(), _expected(n1, gp1, cnt1))
    assert np.array_equal(o2.cpu().numpy(), _expected(n2, None, cnt2))


def test_noalloc_rejects_sizes_beyond_scratch(env):
    torch, sic, h = env
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    n_too_big = MAX_LEN  # n + 1 exceeds the static scratch's 2^26 entries
    code = sic.lib().sic_factor_nnz_noalloc(h.ptr, None, n_too_big, sic._dptr(cnt), n_too_big,
                                            sic._dptr(out), sic._stream(None))
    assert code == sic.SIC_ERR_UNSUPPORTED
