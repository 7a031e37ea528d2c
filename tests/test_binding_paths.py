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
