"""Host logic of bench.py's roofline: which timed products it averages."""
import bench


def test_steady_state_takes_the_modes_kernel_and_its_busiest_width():
    # (ms, work, kind): many small digit-plane products (a norm estimate),
    # split-TF32 products at two widths, a few digit-plane products at the
    # steady width (a refinement tail)
    recs = [(0.05, 6.4e7, 2)] * 70 + [(0.03, 8.08e8, 1)] * 50 + [(0.04, 1.6e9, 1)] * 3 + \
           [(0.09, 8.08e8, 2)] * 20
    n, ms, w = bench.steady_state(recs, bench.MODE_KIND["mixed"])
    assert (n, w) == (50, 8.08e8) and abs(ms - 0.03) < 1e-12
    n, ms, w = bench.steady_state(recs, bench.MODE_KIND["fp64tc"])
    assert (n, w) == (70, 6.4e7)  # by total time: 3.5 ms against 1.8 ms
    n, ms, w = bench.steady_state(recs, bench.MODE_KIND["fp64tc"], 8.08e8)  # the solves' final width
    assert (n, w) == (20, 8.08e8) and abs(ms - 0.09) < 1e-12
    n, ms, w = bench.steady_state(recs, bench.MODE_KIND["fp64"])
    assert n == 0
    n, ms, w = bench.steady_state(recs)
    assert (n, w) == (70, 6.4e7)
