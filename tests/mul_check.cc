// mul_check.cc -- the integer-pipeline binary64 products (fp64_mul.cuh:
// mul_rn_core with a split coefficient, sqr_rn_core) against the host's own
// IEEE multiplication, for the tests.  Built with -ffp-contract=off; the host
// multiplies in binary64, round to nearest even.
#include <cstdint>
#include <cstring>

#include "../paper_1309_1894_gb300/csrc/fp64_mul.cuh"

namespace {

uint64_t bits(double v) {
    uint64_t u;
    std::memcpy(&u, &v, 8);
    return u;
}

}  // namespace

extern "C" {

// For i < n: the fast path's RN(a[i] * b[i]) (square: RN(a[i] * a[i])) and
// its slow flag.  Returns the number of pairs whose fast-path bits differ
// from the host's product; *fast counts the pairs left on the fast path and
// slow_out[i] (when not NULL) records the flag of each pair.
int64_t mul_check(int64_t n, const double *a, const double *b, int square, int64_t *fast,
                  uint8_t *slow_out) {
    int64_t bad = 0, ok = 0;
    for (int64_t i = 0; i < n; ++i) {
        bool slow = false;
        uint64_t r;
        double want;
        if (square) {
            r = wx::sqr_rn_core(bits(a[i]), slow);
            want = a[i] * a[i];
        } else {
            r = wx::mul_rn_core(wx::mul_coef_of(bits(a[i])), bits(b[i]), slow);
            want = a[i] * b[i];
        }
        if (slow_out) slow_out[i] = slow;
        if (slow) continue;
        ++ok;
        bad += r != bits(want);
    }
    *fast = ok;
    return bad;
}

}  // extern "C"
