// serve_ring.h -- slot allocation of the serving loop's pair ring (host only).
//
// Requests hold [off, off + q) of a ring of `cap` slots and leave it in the
// order they entered (FIFO). The live blocks are therefore one run
// [first, end) -- or two once the ring has wrapped (the newest block starts
// below the oldest): [first, cap) and [0, end). A new block of q slots goes at
// `end` if it fits before the next live slot or the ring's end, else at 0 if
// it fits before `first`; the slots skipped at the end when a block wraps to 0
// come free again when the blocks before them leave.
#pragma once

#include <cstdint>

namespace pll {

// empty: no live block; first: start of the oldest; back_off, back_end: start
// and end of the newest. Returns false when no place fits q slots.
inline bool ring_place(bool empty, uint64_t first, uint64_t back_off, uint64_t back_end, uint64_t cap,
                       uint64_t q, uint64_t *off) {
    if (q > cap) return false;
    if (empty) {
        *off = 0;
        return true;
    }
    if (back_off >= first) {  // not wrapped: free [back_end, cap) and [0, first)
        if (cap - back_end >= q) { *off = back_end; return true; }
        if (first >= q) { *off = 0; return true; }
        return false;
    }
    if (first - back_end >= q) { *off = back_end; return true; }  // wrapped: free [back_end, first)
    return false;
}

}  // namespace pll
