"""Byte-count conventions for the bandwidth metric.

Section 4 (Table 1 and the bandwidth paragraph of Section 4.1) reports the
bandwidth of a call as the bytes of mesh data it accesses divided by its time.
For a plain batched solve that is the four coefficient arrays a, b, c, d read
once and the solution written once: 5 words per unknown (20 B in FP32, which
reproduces Table 1: 8000 x 128 x 20 B / 0.47 ms = 43.6 GB/s, printed 43.34).
Accumulating into u (u += x) also reads u: 6 words per unknown.

The ADI step is counted for the schedule that runs, with coefficients
generated in the kernels.  3D: u_new = Z^{-1}(Z u + Y^{-1} X^{-1} d), so
pass A reads u and writes e = Z u + (y-tile values), pass B reads e and writes
u -- 4 words per mesh point (the reduced y values, 2 per 16 points, are not
counted).  2D: pass A reads u and writes w = X^{-1} d, pass B reads w and u
and writes u -- 5 words per mesh point.
"""


def solve_bytes(n_unknowns: int, itemsize: int, accumulate: bool = False) -> int:
    return (6 if accumulate else 5) * int(n_unknowns) * int(itemsize)


def adi_step_bytes(n_points: int, itemsize: int, ndim: int = 3) -> int:
    return (4 if ndim == 3 else 5) * int(n_points) * int(itemsize)


def gbps(nbytes: float, seconds: float) -> float:
    return nbytes / seconds / 1e9
