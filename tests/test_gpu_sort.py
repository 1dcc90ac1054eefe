"""The tree build's hand-written radix sort and prefix scans (the Morton ordering of Sec. 2.5)
against numpy on the same seeded inputs: bit-exact, including the order of equal keys."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_1506_05957_gb300 import binding as B  # noqa: E402


def _to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _keys(n, seed, kind):
    rng = np.random.default_rng(seed)
    if kind == "full":
        k = rng.integers(0, 2**63, size=n, dtype=np.int64).view(np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, size=n, dtype=np.int64).view(np.uint64)
    elif kind == "dups":   # few distinct keys: stability decides the value order
        k = rng.integers(0, 7, size=n).astype(np.uint64) << np.uint64(40)
    elif kind == "equal":
        k = np.full(n, 12345, dtype=np.uint64)
    elif kind == "sorted":
        k = np.sort(rng.integers(0, 2**40, size=n).astype(np.uint64))
    else:                  # reversed
        k = np.sort(rng.integers(0, 2**40, size=n).astype(np.uint64))[::-1].copy()
    return k


@pytest.mark.parametrize("n", [0, 1, 2, 31, 1000, 4097, 123457, 1 << 20])
@pytest.mark.parametrize("kind", ["full", "dups", "equal", "sorted", "reversed"])
def test_sort_pairs_matches_stable_argsort(n, kind):
    k = _keys(n, 17 + n, kind)
    v = np.arange(n, dtype=np.int32)[::-1].copy()
    kd = _to_dev(k.view(np.int64), torch.int64)
    vd = _to_dev(v, torch.int32)
    ko, vo = B.sort_pairs_u64(kd, vd)
    order = np.argsort(k, kind="stable")
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), k[order])
    assert np.array_equal(vo.cpu().numpy(), v[order])
    # the inputs are left unchanged
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), k)


@pytest.mark.parametrize("end_bit", [8, 13, 30, 63])
def test_sort_partial_bits_orders_by_low_bits_only(end_bit):
    n = 50000
    rng = np.random.default_rng(end_bit)
    k = rng.integers(0, 2**62, size=n).astype(np.uint64)
    kd = _to_dev(k.view(np.int64), torch.int64)
    ko, _ = B.sort_pairs_u64(kd, None, end_bit=end_bit)
    # digits are whole bytes: the sort orders by bits [0, 8 ceil(end_bit / 8)), stably
    nb = min(64, 8 * ((end_bit + 7) // 8))
    mask = np.uint64((1 << nb) - 1) if nb < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(k & mask, kind="stable")
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), k[order])


@pytest.mark.parametrize("n", [0, 1, 5, 1023, 1024, 1025, 77777, 3 << 20])
@pytest.mark.parametrize("inclusive", [False, True])
def test_scan_matches_cumsum(n, inclusive):
    rng = np.random.default_rng(n)
    x = rng.integers(-50, 200, size=n).astype(np.int32)
    xd = _to_dev(x, torch.int32)
    out = B.scan_i32(xd, inclusive=inclusive).cpu().numpy()
    ref = np.cumsum(x.astype(np.int64))
    if not inclusive:
        ref = np.concatenate([[0], ref[:-1]]) if n else ref
    assert np.array_equal(out.astype(np.int64), ref)


def test_scan_in_place_and_argument_errors():
    x = _to_dev(np.ones(100000, dtype=np.int32), torch.int32)
    B.scan_i32(x, inclusive=True, out=x)
    assert np.array_equal(x.cpu().numpy(), np.arange(1, 100001, dtype=np.int32))
    k = _to_dev(np.arange(10, dtype=np.int64), torch.int64)
    with pytest.raises(B.FmmBemError):
        B.sort_pairs_u64(k, None, end_bit=65)
    # aliased input and output keys are refused before any device work
    rc = B.lib().fmmbem_sort_pairs_u64(B._vp(k.data_ptr()), B._vp(k.data_ptr()), None, None, 10, 0, None)
    assert rc == B.FMMBEM_EINVAL
