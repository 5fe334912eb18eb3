/*
 * CPU oracle for FDTD-2D (the two-dimensional finite-difference time-domain
 * kernel of the PCOT paper's benchmark suite, Sec. 5.1.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by the test-suite and the benchmark's
 * CPU-baseline arm together with oracle.c; shares no code with the CUDA
 * library, which never calls it.
 *
 * Fields ex, ey, hz: nx x ny values each, row-major with row stride s (>= ny).
 * One time step t, in this order:
 *   ey[0][j]  = fict[t]                                         (all j)
 *   ey[i][j]  = ey[i][j] - 0.5 * (hz[i][j] - hz[i-1][j])        (i >= 1, all j)
 *   ex[i][j]  = ex[i][j] - 0.5 * (hz[i][j] - hz[i][j-1])        (all i, j >= 1)
 *   hz[i][j]  = hz[i][j] - 0.7 * (((ex[i][j+1] - ex[i][j]) + ey[i+1][j]) - ey[i][j])
 *                                                               (i <= nx-2, j <= ny-2)
 * so the electric fields of step t read the magnetic field of step t-1 and
 * the magnetic field reads the electric fields of step t.  Every operation is
 * a separately rounded IEEE-754 binary64 operation in the order written.
 *
 * Parity status: pinned by a hand-derived step (tests/golden/fdtd2d_steps.txt),
 * the exact set of cells one perturbed input changes in one step, the 1-D
 * Yee recurrence that fields constant along j follow away from the right
 * edge, and zero fields with a zero source staying zero.
 */
#include <stdint.h>

int oracle_fdtd2d(int64_t nx, int64_t ny, int64_t s, double *ex, double *ey, double *hz, const double *fict,
                  int64_t T)
{
    if (nx < 1 || ny < 1 || s < ny || !ex || !ey || !hz || (T > 0 && !fict) || T < 0) return -1;
    for (int64_t t = 0; t < T; ++t) {
        for (int64_t j = 0; j < ny; ++j) ey[j] = fict[t];
        for (int64_t i = 1; i < nx; ++i)
            for (int64_t j = 0; j < ny; ++j)
                ey[i * s + j] = ey[i * s + j] - 0.5 * (hz[i * s + j] - hz[(i - 1) * s + j]);
        for (int64_t i = 0; i < nx; ++i)
            for (int64_t j = 1; j < ny; ++j)
                ex[i * s + j] = ex[i * s + j] - 0.5 * (hz[i * s + j] - hz[i * s + j - 1]);
        for (int64_t i = 0; i < nx - 1; ++i)
            for (int64_t j = 0; j < ny - 1; ++j)
                hz[i * s + j] = hz[i * s + j] -
                                0.7 * (((ex[i * s + j + 1] - ex[i * s + j]) + ey[(i + 1) * s + j]) - ey[i * s + j]);
    }
    return 0;
}
