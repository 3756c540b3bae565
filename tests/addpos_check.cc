// addpos_check.cc -- the integer-pipeline sum of two non-negative binary64
// values (fp64_addpos.cuh) against the host's own IEEE addition, for the
// tests.  Built with -ffp-contract=off; the host adds in binary64, round to
// nearest even.
#include <cstdint>
#include <cstring>

#include "../paper_1309_1894_gb300/csrc/fp64_addpos.cuh"

extern "C" {

// Number of pairs whose fast-path result differs bitwise from a + b;
// *fast counts the pairs the fast path took (the others are flagged slow).
int64_t addpos_check(int64_t n, const double *a, const double *b, int64_t *fast) {
    int64_t bad = 0, ok = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t ua, ub;
        std::memcpy(&ua, &a[i], 8);
        std::memcpy(&ub, &b[i], 8);
        bool slow = false;
        const uint64_t r = wx::add_pos_core(ua, ub, slow);
        if (slow) continue;
        ++ok;
        const double want = a[i] + b[i];
        uint64_t uw;
        std::memcpy(&uw, &want, 8);
        bad += r != uw;
    }
    *fast = ok;
    return bad;
}

}  // extern "C"
