/*
 * Oracle: the exact per-baseline aperture kernel of a pair of uniform disks
 * with different pointing offsets, and FP64 degridding with it.
 * TEST INFRASTRUCTURE ONLY -- called from the Python oracle (oracle/exact.py),
 * never from the product library, and sharing no code with it.
 *
 * Paper basis (Bhatnagar & Cornwell 2017): Sec. 3 writes A_ij as the
 * transform of the baseline's primary beam E_i E_j with E_i the antenna's
 * pattern shifted by its offset, models the main lobe as a Gaussian (Eq.
 * AIJPOINTING: A° times a decorrelation factor times a phase ramp) and notes
 * that a more accurate pattern may replace the Gaussian.  Here E is the
 * uniform disk's own pattern.  With aperture a(w) (1 inside radius R =
 * D_lambda / 2) and E(l) its transform, the transform of E(l-l_i) E(l-l_j) is
 *
 *   A_ij(du) = exp(i pi du.(l_i + l_j)) * O(du; dl) / (pi R^2)^2,
 *   O(du; dl) = integral over the lens {|w - du/2| <= R, |w + du/2| <= R}
 *               of cos(2 pi w.dl) d^2w,              dl = l_i - l_j,
 *
 * (substitute w = w1 - du/2 in the autocorrelation of the two shifted
 * apertures; the lens is symmetric under w -> -w, so only the cosine
 * survives).  At dl = 0, O is the overlap area and A_ij is A° times the ramp;
 * the Gaussian factor of Eq. AIJPOINTING approximates O's dependence on dl.
 *
 * Quadrature.  In the frame e_par = du/|du|, e_perp, write a = dl.e_par,
 * b = dl.e_perp, rho = |du|.  The inner integral over w_perp in [-h, h] is
 * closed: int cos(2 pi b w) dw = 2 sin(k h)/k, k = 2 pi b; its b-derivative
 * is int -2 pi w sin(k w) dw.  The outer integral over w_par in [0, R - rho/2]
 * (times 2: the integrand is even) uses w_par + rho/2 = R cos(theta),
 * h = R sin(theta), theta in [0, acos(rho / 2R)], which makes the integrand
 * smooth, and Gauss-Legendre with kNodes nodes in theta.
 *
 * Degridding follows the table rule of the radial kernel (oracle/aperture.py):
 * a tap at rho cells reads t = rho ov, n = floor(t), f = t - n, and takes
 * (1-f) K(n) + f K(n+1), where K(n) is the exact kernel at radius n / ov
 * cells in the tap's own direction (zero when n + 1 >= len).
 */
#include <math.h>
#include <stddef.h>

#define kNodes 32

static double gl_x[kNodes], gl_w[kNodes];
static int gl_ready = 0;

/* Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n from
 * the Chebyshev-like initial guesses cos(pi (k + 3/4) / (n + 1/2)), P_n and
 * P_n' from the three-term recurrence, w = 2 / ((1 - x^2) P_n'(x)^2). */
static void gl_init(void) {
    const double pi = 3.14159265358979323846;
    const int n = kNodes;
    for (int k = 0; k < n; ++k) {
        double x = cos(pi * (k + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[k] = x;
        gl_w[k] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

/* 2 sin(k h) / k (the integral of cos(k w) over [-h, h]) and its derivative
 * with respect to b = k / (2 pi): int_{-h}^{h} -2 pi w sin(k w) dw.  Series
 * in x = k h below |x| = 0.5 (both are even / odd in k with no cancellation
 * problem there), closed forms above. */
static void inner(double k, double h, double *I, double *Ib) {
    const double pi = 3.14159265358979323846;
    const double x = k * h;
    if (fabs(x) < 0.5) {
        /* sin(x)/x = sum (-1)^n x^2n / (2n+1)!;
           int_{-h}^{h} w sin(k w) dw = 2 h^2 sum (-1)^n x^(2n+1) / ((2n+1)! (2n+3)) */
        double s = 0.0, t = 0.0, term = 1.0;       /* term = (-1)^n x^2n / (2n+1)! */
        for (int n = 0; n < 12; ++n) {
            s += term;
            t += term / (2.0 * n + 3.0);
            term *= -x * x / ((2.0 * n + 2.0) * (2.0 * n + 3.0));
        }
        *I = 2.0 * h * s;
        *Ib = -2.0 * pi * 2.0 * h * h * x * t;
    } else {
        *I = 2.0 * sin(x) / k;
        *Ib = -2.0 * pi * 2.0 * (sin(x) / (k * k) - h * cos(x) / k);
    }
}

/* O(rho; a, b) and its derivatives dO/da, dO/db for disks of radius R
 * (rho, R in wavelengths; a, b in radians). */
static void overlap(double rho, double a, double b, double R, double *O, double *Oa, double *Ob) {
    const double pi = 3.14159265358979323846;
    *O = *Oa = *Ob = 0.0;
    if (rho >= 2.0 * R) return;
    const double th0 = acos(rho / (2.0 * R));
    const double k = 2.0 * pi * b;
    double so = 0.0, sa = 0.0, sb = 0.0;
    for (int q = 0; q < kNodes; ++q) {
        const double th = 0.5 * th0 * (gl_x[q] + 1.0);
        const double wq = 0.5 * th0 * gl_w[q];
        const double wpar = R * cos(th) - 0.5 * rho;
        const double h = R * sin(th);
        const double jac = R * sin(th);            /* dw_par = R sin(theta) dtheta */
        double I, Ib;
        inner(k, h, &I, &Ib);
        const double ca = cos(2.0 * pi * a * wpar), sna = sin(2.0 * pi * a * wpar);
        so += wq * jac * ca * I;
        sa += wq * jac * (-2.0 * pi * wpar * sna) * I;
        sb += wq * jac * ca * Ib;
    }
    *O = 2.0 * so;
    *Oa = 2.0 * sa;
    *Ob = 2.0 * sb;
}

void oracle_exact_overlap(long n, const double *rho, const double *a, const double *b, double R,
                          double *O, double *Oa, double *Ob) {
    if (!gl_ready) gl_init();
    for (long i = 0; i < n; ++i) overlap(rho[i], a[i], b[i], R, O + i, Oa + i, Ob + i);
}

/*
 * Per-visibility sums with the exact kernel, over the S x S tap window (same
 * window and cell-offset convention as oracle/degrid.c):
 *   T0 = sum_g K G_g ramp,  Tu = sum_g du_g K G_g ramp,  Tv = sum_g dv_g K G_g ramp,
 *   TX = sum_g dK/d(dl_x) G_g ramp,  TY = sum_g dK/d(dl_y) G_g ramp,
 * ramp = exp(i pi (du_g L + dv_g M)), K the interpolated exact kernel times
 * du^2 / (pi R^2)^2 (the radial table's normalisation), (dl_x, dl_y) =
 * (l_i - l_j, m_i - m_j) of the visibility's baseline, R = D_lambda / 2 of its
 * channel, len the channel's table length.
 */
void oracle_exact_degrid(long n_vis,
                         const double *u, const double *v,       /* [n_vis] wavelengths */
                         const double *L, const double *M,       /* [n_vis] l_i+l_j, m_i+m_j */
                         const double *dlx, const double *dly,   /* [n_vis] l_i-l_j, m_i-m_j */
                         const double *R, const int *len,        /* [n_vis] disk radius (wavelengths), table length */
                         int ov, const double *grid, int ng, double du, int support,
                         double *t0, double *tu, double *tv, double *tx, double *ty) {
    const double pi = 3.14159265358979323846;
    if (!gl_ready) gl_init();
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < n_vis; ++k) {
        const double x = u[k] / du + 0.5 * ng;
        const double y = v[k] / du + 0.5 * ng;
        const long x0 = (long)floor(x) - support / 2 + 1;
        const long y0 = (long)floor(y) - support / 2 + 1;
        const double area = pi * R[k] * R[k];
        const double norm = du * du / (area * area);
        double s[10] = {0};
        for (int bb = 0; bb < support; ++bb) {
            const long gy = y0 + bb;
            if (gy < 0 || gy >= ng) continue;
            const double dv = (y - (double)gy) * du;
            for (int aa = 0; aa < support; ++aa) {
                const long gx = x0 + aa;
                if (gx < 0 || gx >= ng) continue;
                const double duu = (x - (double)gx) * du;
                const double rw = sqrt(duu * duu + dv * dv);     /* wavelengths */
                const double t = rw / du * ov;
                const long n = (long)floor(t);
                if (n + 1 >= len[k]) continue;
                const double f = t - (double)n;
                /* tap direction (any unit vector at the origin: the lens is a disk there) */
                const double ex = rw > 0.0 ? duu / rw : 1.0, ey = rw > 0.0 ? dv / rw : 0.0;
                const double a = dlx[k] * ex + dly[k] * ey;
                const double b = -dlx[k] * ey + dly[k] * ex;     /* e_perp = (-ey, ex) */
                double O0, Oa0, Ob0, O1, Oa1, Ob1;
                overlap((double)n * du / ov, a, b, R[k], &O0, &Oa0, &Ob0);
                overlap((double)(n + 1) * du / ov, a, b, R[k], &O1, &Oa1, &Ob1);
                const double Ov = ((1.0 - f) * O0 + f * O1) * norm;
                const double Oav = ((1.0 - f) * Oa0 + f * Oa1) * norm;
                const double Obv = ((1.0 - f) * Ob0 + f * Ob1) * norm;
                /* gradient in (dl_x, dl_y): dO/da e_par + dO/db e_perp */
                const double gxv = Oav * ex - Obv * ey;
                const double gyv = Oav * ey + Obv * ex;
                const double ph = pi * (duu * L[k] + dv * M[k]);
                const double cr = cos(ph), ci = sin(ph);
                const double gr = grid[2 * (gy * ng + gx)], gi = grid[2 * (gy * ng + gx) + 1];
                const double zr = cr * gr - ci * gi, zi = cr * gi + ci * gr;   /* ramp * G */
                s[0] += Ov * zr;        s[1] += Ov * zi;
                s[2] += duu * Ov * zr;  s[3] += duu * Ov * zi;
                s[4] += dv * Ov * zr;   s[5] += dv * Ov * zi;
                s[6] += gxv * zr;       s[7] += gxv * zi;
                s[8] += gyv * zr;       s[9] += gyv * zi;
            }
        }
        t0[2 * k] = s[0]; t0[2 * k + 1] = s[1];
        tu[2 * k] = s[2]; tu[2 * k + 1] = s[3];
        tv[2 * k] = s[4]; tv[2 * k + 1] = s[5];
        tx[2 * k] = s[6]; tx[2 * k + 1] = s[7];
        ty[2 * k] = s[8]; ty[2 * k + 1] = s[9];
    }
}
