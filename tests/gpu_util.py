"""GPU test helpers: guarded device buffers and bitwise comparison.

Each vector lives inside its own allocation with guard regions of a canary
bit pattern before and after it; ``Guarded.check()`` asserts the guards are
untouched.  compute-sanitizer is not used, so the guards are the out-of-bounds
check.  Comparisons are on the 64-bit patterns (0 ULP).
"""
import numpy as np
import torch

# A signalling-NaN bit pattern the method never produces from finite inputs.
CANARY = 0x7FF4DEADBEEFCAFE
CANARY_I64 = CANARY - (1 << 64) if CANARY >= (1 << 63) else CANARY
GUARD = 512  # elements (4 KiB) on each side


class Guarded:
    """A length-n float64 view at byte offset ``off`` (a multiple of 8) inside a
    256-byte-aligned allocation framed by canary guards."""

    def __init__(self, n: int, off: int = 0, device="cuda"):
        assert off % 8 == 0
        self.n, self.o = n, off // 8
        self.buf = torch.empty(GUARD + self.o + n + GUARD, dtype=torch.float64, device=device)
        assert self.buf.data_ptr() % 256 == 0
        self.buf.view(torch.int64).fill_(CANARY_I64)
        self.t = self.buf[GUARD + self.o: GUARD + self.o + n]

    def set(self, host: np.ndarray):
        self.t.copy_(torch.from_numpy(np.ascontiguousarray(host)))
        return self

    def check(self):
        b = self.buf.view(torch.int64)
        lo = b[: GUARD + self.o]
        hi = b[GUARD + self.o + self.n:]
        assert bool((lo == CANARY_I64).all()), "guard before the vector was overwritten"
        assert bool((hi == CANARY_I64).all()), "guard after the vector was overwritten"


def bits_equal(dev: torch.Tensor, host: np.ndarray) -> tuple[bool, str]:
    """Bitwise equality of a device float64 tensor and a host array."""
    got = dev.detach().cpu().numpy().view(np.uint64)
    want = np.ascontiguousarray(host, dtype=np.float64).view(np.uint64)
    if got.shape != want.shape:
        return False, f"shape {got.shape} vs {want.shape}"
    bad = np.nonzero(got != want)[0]
    if bad.size == 0:
        return True, ""
    i = int(bad[0])
    return False, (f"{bad.size} mismatches, first at {i}: got "
                   f"{float(got[i:i+1].view(np.float64)[0]).hex()} want "
                   f"{float(want[i:i+1].view(np.float64)[0]).hex()}")


def dev_bits_equal(a: torch.Tensor, b: torch.Tensor) -> bool:
    return bool(torch.equal(a.view(torch.int64), b.view(torch.int64)))
