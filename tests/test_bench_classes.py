"""The class rows of the benchmark's sweep (alias and mixed-offset cases at
n = 2^24, 2^26, 2^28) are timed by the step's own rule: a call expected under
200 us runs as a batch of calls on disjoint slices.  On the CPU, with made-up
addresses: each call keeps the row's alias relation and byte offsets, the
slices of a batch never overlap, and every access stays inside the buffers
the benchmark allocates (2^28 + 11 doubles each)."""
import pytest

import bench

NUMEL = (1 << 28) + 3 + 8
BASE = {"x": 1 << 40, "y": 2 << 40, "w": 3 << 40}  # 256-byte aligned, far apart


def spans(calls, n, alias):
    out = []
    for a, b, c in calls:
        out += [(a, a + 8 * n), (c, c + 8 * n)]
        if alias != "x=y":
            out.append((b, b + 8 * n))
    return out


@pytest.mark.parametrize("k", [24, 26, 28])
@pytest.mark.parametrize("case", bench.CLASS_CASES, ids=[c[0] for c in bench.CLASS_CASES])
def test_class_batch(k, case):
    name, ox, oy, ow, alias = case
    n = 1 << k
    calls = bench.class_batch(BASE["x"], BASE["y"], BASE["w"], NUMEL, n, ox, oy, ow, alias)
    assert len(calls) == bench.flushed_batch(n)
    assert (len(calls) > 1) == (k == 24)  # short calls only are batched
    for a, b, c in calls:
        assert a % 256 == ox and (alias == "x=y" or b % 256 == oy)
        if alias == "w=x":
            assert c == a
        elif alias == "w=y":
            assert c == b
        elif alias == "x=y":
            assert b == a and c % 256 == ow
        else:
            assert len({a, b, c}) == 3 and c % 256 == ow
        for p, key in ((a, "x"), (b, "x" if alias == "x=y" else "y"),
                       (c, {"w=x": "x", "w=y": "y"}.get(alias, "w"))):
            assert BASE[key] <= p and p + 8 * n <= BASE[key] + 8 * NUMEL  # inside its buffer
    # calls of a batch touch disjoint memory (each slice is cold after the flush)
    per_call = [spans([cl], n, alias) for cl in calls]
    for i in range(len(calls)):
        for j in range(i + 1, len(calls)):
            for lo1, hi1 in per_call[i]:
                for lo2, hi2 in per_call[j]:
                    assert hi1 <= lo2 or hi2 <= lo1


def test_class_batch_refuses_slices_past_the_buffer():
    with pytest.raises(AssertionError):
        bench.class_batch(BASE["x"], BASE["y"], BASE["w"], (1 << 24) + 100, 1 << 24, 0, 8, 24,
                          "distinct")
