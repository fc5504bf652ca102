/*
 * Oracle: FP64 degridding with the pointing-modified aperture kernel.
 * TEST INFRASTRUCTURE ONLY -- called from the Python oracle (oracle/degrid.py),
 * never from the product library, and sharing no code with it.
 *
 * Paper basis (Bhatnagar & Cornwell 2017):
 *   Eq. AIJPOINTING:  A_ij(du) = A°(du) [exp(-(l_i-l_j)^2 alpha^2 / 2)] exp(i pi du (l_i + l_j))
 *   Eq. DAIJPOINTING: dA_ij/dl_i = A_ij [(l_j - l_i) alpha^2 + i pi du]
 *   Algorithm 1:      V^M = A_ij * V°, grad V^M = grad A_ij * V° (A-Projection degridding)
 * where du is the kernel's own argument (the Fourier conjugate of l), i.e. the
 * offset between the visibility's uv point and a grid cell.
 *
 * For visibility k with uv point (u_k, v_k) in wavelengths this file returns
 * the three sums, taken over the S x S tap window T(k):
 *     T0 = sum_g  A°(|d_g|) exp(i pi (du_g L + dv_g M)) G_g
 *     Tu = sum_g  du_g * (same term)
 *     Tv = sum_g  dv_g * (same term)
 * with d_g = (u_k - u_g, v_k - v_g), L = l_i + l_j, M = m_i + m_j.  The
 * decorrelation factor and the derivative combinations are applied in Python.
 *
 * Tap window: grid coordinate x = u_k / du + Ng/2; x0 = floor(x) - S/2 + 1;
 * taps x0 .. x0+S-1 (same for y).  Cells outside [0, Ng) contribute nothing.
 * A°(rho) comes from a radial table at `ov` samples per cell with linear
 * interpolation: t = rho*ov, n = floor(t), f = t - n,
 * A = (1-f) tab[n] + f tab[n+1] if n+1 < len, else 0.
 */
#include <math.h>
#include <stddef.h>

void oracle_degrid(long n_vis,
                   const double *u, const double *v,       /* [n_vis] wavelengths */
                   const double *L, const double *M,       /* [n_vis] l_i+l_j, m_i+m_j (rad) */
                   const int *tab_id,                       /* [n_vis] which table */
                   const double *tabs, const long *tab_off, const int *tab_len,
                   int ov,
                   const double *grid,                      /* complex [ng][ng], interleaved re,im */
                   int ng, double du, int support,
                   double *t0, double *tu, double *tv)      /* complex [n_vis], interleaved */
{
    const double pi = 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 64)
    for (long k = 0; k < n_vis; ++k) {
        const double *tab = tabs + tab_off[tab_id[k]];
        const int len = tab_len[tab_id[k]];
        const double x = u[k] / du + 0.5 * ng;
        const double y = v[k] / du + 0.5 * ng;
        const long x0 = (long)floor(x) - support / 2 + 1;
        const long y0 = (long)floor(y) - support / 2 + 1;
        double s0r = 0, s0i = 0, sur = 0, sui = 0, svr = 0, svi = 0;
        for (int b = 0; b < support; ++b) {
            const long gy = y0 + b;
            if (gy < 0 || gy >= ng) continue;
            const double dv = (y - (double)gy) * du;          /* v_k - v_g */
            for (int a = 0; a < support; ++a) {
                const long gx = x0 + a;
                if (gx < 0 || gx >= ng) continue;
                const double duu = (x - (double)gx) * du;     /* u_k - u_g */
                const double rho = sqrt(duu * duu + dv * dv) / du;   /* cells */
                const double t = rho * ov;
                const long n = (long)floor(t);
                if (n + 1 >= len) continue;
                const double f = t - (double)n;
                const double amp = (1.0 - f) * tab[n] + f * tab[n + 1];
                const double ph = pi * (duu * L[k] + dv * M[k]);
                const double kr = amp * cos(ph), ki = amp * sin(ph);
                const double gr = grid[2 * (gy * ng + gx)], gi = grid[2 * (gy * ng + gx) + 1];
                const double pr = kr * gr - ki * gi, pi_ = kr * gi + ki * gr;
                s0r += pr;        s0i += pi_;
                sur += duu * pr;  sui += duu * pi_;
                svr += dv * pr;   svi += dv * pi_;
            }
        }
        t0[2 * k] = s0r; t0[2 * k + 1] = s0i;
        tu[2 * k] = sur; tu[2 * k + 1] = sui;
        tv[2 * k] = svr; tv[2 * k + 1] = svi;
    }
}
