"""Host-side guard of the Paths binding: the C object borrows its index's
device arrays, so using it after the index (or itself) is closed raises
before any call reaches the library."""
import pytest

from paper_1304_4661_gb300 import pll


class _ClosedIndex:
    _h = None


def test_paths_after_index_closed_raises():
    p = pll.Paths.__new__(pll.Paths)
    p.index = _ClosedIndex()
    p._h = 1234
    with pytest.raises(RuntimeError):
        p.parents()
    with pytest.raises(RuntimeError):
        p.offsets([], [])
    with pytest.raises(RuntimeError):
        p.query([], [])
    p._h = None  # nothing to free


def test_index_close_refused_while_borrowed():
    ix = pll.Index.__new__(pll.Index)
    pll.Index.__init__(ix, 1234, 3, 0)  # a handle that is never passed to the library

    class _User:
        _h = 1

    u = _User()
    ix._lend(u)
    with pytest.raises(RuntimeError):
        ix.close()
    u._h = None  # the borrower closed: close() would now free the handle
    ix._h = None  # but this one is fake, so drop it instead
