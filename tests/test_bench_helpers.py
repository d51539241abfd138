"""Host-side helpers of bench.py that need no GPU."""
import bench


def seven_smooth(v):
    for p in (2, 3, 5, 7):
        while v % p == 0:
            v //= p
    return v == 1


def test_smooth7_is_the_nearest_seven_smooth_integer():
    for n in range(1, 400):
        s = bench.smooth7(n)
        assert seven_smooth(s)
        # no 7-smooth integer strictly closer to n
        assert not any(seven_smooth(v) for v in range(max(1, n - abs(s - n) + 1), n + abs(s - n)))
