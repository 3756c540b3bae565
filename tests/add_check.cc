// add_check.cc -- the integer-pipeline binary64 sum of any two values
// (fp64_emu.cuh: add_rn_with, the sum the single-call kernels move off the
// FP64 pipeline) against the host's own IEEE addition, for the tests.  Built
// with -ffp-contract=off; the host adds in binary64, round to nearest even.
#include <cstdint>
#include <cstring>

#include "../paper_1309_1894_gb300/csrc/fp64_emu.cuh"

namespace {

// Stands in for the hardware instruction: records that the integer path
// left the pair out.
struct Leave {
    bool *slow;
    uint64_t operator()(uint64_t, uint64_t) const {
        *slow = true;
        return 0;
    }
};

}  // namespace

extern "C" {

// Number of pairs whose fast-path bits differ from a[i] + b[i]; *fast counts
// the pairs left on the fast path and slow_out[i] records each pair's flag.
int64_t add_check(int64_t n, const double *a, const double *b, int64_t *fast, uint8_t *slow_out) {
    int64_t bad = 0, ok = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t ua, ub;
        std::memcpy(&ua, &a[i], 8);
        std::memcpy(&ub, &b[i], 8);
        bool slow = false;
        const uint64_t r = wx::add_rn_with(ua, ub, Leave{&slow});
        slow_out[i] = slow;
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
