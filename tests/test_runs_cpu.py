"""Run-length encoding of the device neighbour table (host only, through the C ABI).

The pull step of Section 2.2's sparse method finds every neighbour through an index
table: 18 entries per fluid site, as many bytes per update as the 16-bit populations
themselves.  In rows ordering the entries of consecutive sites differ by constant
offsets over most of an x-row, so the table is also kept as runs (per site one word
flagging its non-fluid links and naming its run, per run 18 offsets).  Checked here:

  * decoding the encoding with numpy gives back every entry of the table, for both
    schemes' virtual indices, tables in rows, bricks-like and Morton order, a stride
    larger than the site count, site counts below and across 1024-site chunks, and
    fluid entries beyond the encoded sites (the ghosts of a split partition);
  * a rows-ordered vessel tree compresses (runs of tens of sites); a random order does
    not, and the encoder then reports no encoding; a table of more than 2^20 sites is
    encoded in spans whose runs join up in order;
  * an entry that is neither a fluid index nor the scheme's virtual index, and bad
    arguments, are refused.

The device tables are built here from the canonical table of hg_build_neighbours,
permuted to a lexicographic order in numpy, independently of the library's orderings.
"""
import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S


def _opp(i):
    return i + 1 if i % 2 == 1 else i - 1


def _device_table(xs, nbr_c, order, scheme, stride):
    """Device table in the given site order: fluid entries renumbered, every other entry
    the scheme's virtual index q + dd np."""
    n = xs.shape[0]
    dev_of = np.empty(n, np.int64)
    dev_of[order] = np.arange(n)
    T = np.zeros((18, stride), np.int64)
    q = np.arange(n)
    for i in range(1, 19):
        v = nbr_c[i - 1, order].astype(np.int64)
        dd = (i - _opp(i)) if scheme == "aa" else (_opp(i) - i)
        T[i - 1, :n] = np.where(v >= 0, dev_of[np.maximum(v, 0)], q + dd * stride)
    return T.astype(np.int32)


def _decode(lword, run0, rdelta, n, stride, scheme):
    q = np.arange(n)
    run = run0[q >> 10] + (lword[:n] >> 18).astype(np.int64)
    out = np.zeros((18, n), np.int64)
    for i in range(1, 19):
        dd = (i - _opp(i)) if scheme == "aa" else (_opp(i) - i)
        miss = (lword[:n] >> (i - 1)) & 1
        out[i - 1] = np.where(miss == 1, q + dd * stride, q + rdelta[run, i - 1])
    return out


def _rows_order(xs):
    return np.lexsort((xs[:, 0], xs[:, 1], xs[:, 2]))


def _bricks_like_order(xs):
    b = xs // np.array([16, 4, 4])
    return np.lexsort((xs[:, 0], xs[:, 1], xs[:, 2], b[:, 0], b[:, 1], b[:, 2]))


@pytest.mark.parametrize("scheme", ["ab", "aa"])
@pytest.mark.parametrize("order_name", ["rows", "bricks", "morton"])
def test_decode_equals_table(hemegb_lib, scheme, order_name):
    geo = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7), inlet_speed=0.05, period=200.0)
    xs, nbr_c = hemegb_lib.build_neighbours(geo.xyz, geo.iolets)
    n = xs.shape[0]
    order = {"rows": _rows_order, "bricks": _bricks_like_order, "morton": lambda x: np.arange(len(x))}[order_name](xs)
    stride = (n + 127) // 128 * 128 + 128                       # padding beyond the sites
    T = _device_table(xs, nbr_c, order, scheme, stride)
    enc = hemegb_lib.encode_runs(T, n=n, scheme=scheme)
    if order_name == "rows":
        assert enc is not None
    if enc is None:
        return
    lword, run0, rdelta = enc
    assert np.array_equal(_decode(lword, run0, rdelta, n, stride, scheme), T[:, :n].astype(np.int64))
    assert (lword[:n] >> 28).max() == 0                          # the word uses 28 bits
    assert rdelta.shape[0] * 72 <= 16 * n                        # it saves traffic
    if order_name == "rows":
        assert n / rdelta.shape[0] > 8                           # runs span most of a row


def test_rows_tree_compresses_and_small_tables(hemegb_lib):
    """A 3-D tube in rows order: few runs; prefixes of it (below one chunk, across chunks)
    decode too."""
    geo = S.cylinder(radius=9, length=60)
    xs, nbr_c = hemegb_lib.build_neighbours(geo.xyz, geo.iolets)
    order = _rows_order(xs)
    n_all = xs.shape[0]
    T = _device_table(xs, nbr_c, order, "ab", n_all)
    lword, run0, rdelta = hemegb_lib.encode_runs(T, scheme="ab")
    assert n_all / rdelta.shape[0] > 10
    for n in (700, 1024, 1025, 3000):
        enc = hemegb_lib.encode_runs(T, n=n, n_ref=n_all, scheme="ab")  # entries beyond n: ghosts
        assert enc is not None, n
        assert np.array_equal(_decode(*enc, n, n_all, "ab"), T[:, :n].astype(np.int64)), n


def test_spans_of_a_large_table(hemegb_lib):
    """More than 2^20 sites: the encoder works on spans of 2^20 sites in parallel, each
    starting a run; the decode is still every entry, and run0 follows the spans' offsets."""
    geo = S.cylinder(radius=30, length=420)
    xs, nbr_c = hemegb_lib.build_neighbours(geo.xyz, geo.iolets)
    n = xs.shape[0]
    assert n > (1 << 20)
    stride = (n + 127) // 128 * 128
    T = _device_table(xs, nbr_c, _rows_order(xs), "aa", stride)
    lword, run0, rdelta = hemegb_lib.encode_runs(T, n=n, scheme="aa")
    assert np.array_equal(_decode(lword, run0, rdelta, n, stride, "aa"), T[:, :n].astype(np.int64))
    q = np.arange(n)
    run = run0[q >> 10] + (lword[:n] >> 18).astype(np.int64)
    assert run[0] == 0 and run[-1] == rdelta.shape[0] - 1 and np.all(np.diff(run) >= 0)
    assert run[1 << 20] == run[(1 << 20) - 1] + 1                 # a span starts a run


def test_random_order_does_not_compress(hemegb_lib):
    geo = S.cylinder(radius=6, length=30)
    xs, nbr_c = hemegb_lib.build_neighbours(geo.xyz, geo.iolets)
    order = np.random.default_rng(5).permutation(xs.shape[0])
    T = _device_table(xs, nbr_c, order, "aa", xs.shape[0])
    assert hemegb_lib.encode_runs(T, scheme="aa") is None


def test_bad_entries_and_arguments(hemegb_lib):
    geo = S.cylinder(radius=6, length=30)
    xs, nbr_c = hemegb_lib.build_neighbours(geo.xyz, geo.iolets)
    n = xs.shape[0]
    T = _device_table(xs, nbr_c, _rows_order(xs), "ab", n)
    assert hemegb_lib.encode_runs(T, scheme="ab") is not None
    assert hemegb_lib.encode_runs(T, scheme="aa") is None      # virtual indices of the other scheme
    q = int(np.argmax((T[0] < 0) | (T[0] >= n)))                # a site with a non-fluid +x link
    bad = T.copy()
    bad[0, q] += 1                                              # neither fluid nor virtual
    assert hemegb_lib.encode_runs(bad, scheme="ab") is None
    with pytest.raises(hemegb_lib.HgError):
        hemegb_lib.encode_runs(T, n=n, n_ref=n - 1, scheme="ab")   # n_ref below n
    with pytest.raises(hemegb_lib.HgError):
        hemegb_lib.encode_runs(T, scheme=7)
