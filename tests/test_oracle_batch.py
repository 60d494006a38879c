"""Pins of the oracle's ragged-batch entry point ``perm_batch`` (the checker of
the full-size ragged parity test and the timed CPU baseline).

``perm_batch`` only reads the packed layout (base matrices at element offsets,
multiplicities at entry offsets) and deals items to host threads; the
arithmetic is ``perm_ryser`` of each item.  So every item of a batch must
equal a single-threaded ``perm_ryser`` call on that item bit for bit, in both
modes, whatever the thread count.  The batches here are laid out so that a
slip in the offset handling cannot go unnoticed: items are stored out of
order, with gaps between them filled with NaN matrix entries and with
multiplicities that break sum r = sum c, and row and column offsets differ
from each other and from the matrix offsets."""
import math

import numpy as np
import pytest

import oracle as O


def crandn(k, l, rng):
    return (rng.standard_normal((k, l)) + 1j * rng.standard_normal((k, l))) / math.sqrt(2 * max(k, l, 1))


def parts(n, rng, maxpart=3):
    out, left = [], n
    while left:
        p = min(int(rng.integers(1, maxpart + 1)), left)
        out.append(p)
        left -= p
    return out


def mixed_items(rng):
    items = []
    items.append((np.zeros((0, 0), dtype=complex), [], []))              # n = 0, empty base
    items.append((crandn(2, 3, rng), [0, 0], [0, 0, 0]))                 # n = 0, zero multiplicities
    items.append((crandn(5, 1, rng), [1] * 5, [5]))                      # tall base
    items.append((crandn(1, 4, rng), [4], [1] * 4))                      # wide base
    items.append((crandn(4, 5, rng), [2, 0, 1, 0], [0, 1, 0, 2, 0]))     # zero rows and columns
    items.append((crandn(1, 1, rng), [1], [1]))                          # n = 1
    items.append((crandn(16, 16, rng), [1] * 16, [1] * 16))              # 2^16 Ryser terms
    for _ in range(14):
        n = int(rng.integers(2, 13))
        r, c = parts(n, rng), parts(n, rng)
        items.append((crandn(len(r), len(c), rng), r, c))
    return items


def scattered_layout(items, rng):
    """Packed arrays with the items in a shuffled storage order and gaps of
    poison between them: NaN matrix entries and multiplicities of 7."""
    order = rng.permutation(len(items))
    mats, rm, cm = [], [], []
    mat_off = np.zeros(len(items), dtype=np.int64)
    row_off = np.zeros(len(items), dtype=np.int64)
    col_off = np.zeros(len(items), dtype=np.int64)
    mo = ro = co = 0
    for b in order:
        B, r, c = items[b]
        gm, gr, gc = (int(x) for x in rng.integers(1, 5, 3))
        mats.append(np.full(gm, complex(np.nan, np.nan)))
        rm.append(np.full(gr, 7, dtype=np.int32))
        cm.append(np.full(gc + 1, 7, dtype=np.int32))  # column gaps differ from row gaps
        mo += gm
        ro += gr
        co += gc + 1
        mat_off[b], row_off[b], col_off[b] = mo, ro, co
        mats.append(np.asarray(B, dtype=complex).reshape(-1))
        rm.append(np.asarray(r, dtype=np.int32))
        cm.append(np.asarray(c, dtype=np.int32))
        mo += B.size
        ro += len(r)
        co += len(c)
    mats.append(np.full(3, complex(np.nan, np.nan)))
    k = np.array([B.shape[0] for B, _, _ in items], dtype=np.int32)
    l = np.array([B.shape[1] for B, _, _ in items], dtype=np.int32)
    return (np.concatenate(mats), mat_off, k, l, np.concatenate(rm), row_off,
            np.concatenate(cm), col_off)


@pytest.mark.parametrize("gold", [False, True])
@pytest.mark.parametrize("nthreads", [1, 3, 64])
def test_batch_equals_single_item_calls_bit_for_bit(gold, nthreads):
    rng = np.random.default_rng(2024 + nthreads)
    items = mixed_items(rng)
    layout = scattered_layout(items, rng)
    per, sabs, bound = O.perm_batch(*layout, gold=gold, nthreads=nthreads, info=True)
    assert len(items) < 64  # the last case runs more threads than items
    for b, (B, r, c) in enumerate(items):
        p1, s1, b1 = O.perm_ryser(B, r, c, gold=gold, nthreads=1, info=True)
        assert per[b] == p1, (b, per[b], p1)
        assert sabs[b] == s1 and bound[b] == b1, b
    # the trivial items and a closed form, independently of perm_ryser
    assert per[0] == 1.0 and per[1] == 1.0
    B, r, c = items[5]
    assert per[5] == B[0, 0]


def test_batch_reads_rows_and_columns_from_their_own_offsets():
    """An item whose row and column multiplicities differ (a tall base): the
    result must be per(B repeated by c) with the column multiplicity applied
    to the column, which a swapped offset would turn into an argument error or
    another value."""
    rng = np.random.default_rng(77)
    B = crandn(3, 1, rng)
    items = [(B, [1, 1, 1], [3]), (crandn(2, 2, rng), [1, 1], [1, 1])]
    layout = scattered_layout(items, rng)
    per = O.perm_batch(*layout, nthreads=2)
    # per of the 3 x 3 matrix whose columns all equal B[:, 0]: 3! * prod B_i0
    want = math.factorial(3) * np.prod(B[:, 0])
    assert abs(per[0] - want) <= 1e-14 * abs(want)


def test_batch_rejects_inconsistent_item():
    rng = np.random.default_rng(78)
    items = [(crandn(2, 2, rng), [1, 1], [1, 1]), (crandn(2, 2, rng), [1, 2], [1, 1])]
    with pytest.raises(ValueError):
        O.perm_batch(*scattered_layout(items, rng), nthreads=2)
