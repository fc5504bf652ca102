// A-priori aperture kernel A° as radial tables, one per channel (Algorithm 1,
// second pre-compute; Sec. 3: A°_ij holds the pointing-free part of A_ij).
//
// Uniform disk of diameter D (D_lambda = D nu / c): A°(q) is the overlap area
// of two disks of radius R = D_lambda / 2 whose centres are q apart, divided
// by (pi R^2)^2 -- the Fourier transform of the Airy power beam, integral 1.
// Gaussian voltage pattern exp(-alpha^2 rho^2): A°(q) = (pi / 2 alpha^2)
// exp(-pi^2 q^2 / (2 alpha^2)).
// Caller's table T (PSC_AP_TABLE): A°(q) = T(q / D_lambda) / D_lambda^2 with T
// linear between its samples at x = k / (len - 1), and 0 from q = D_lambda on.
// Entry n holds (A°(n du / ov) du^2, A°((n+1) du / ov) du^2 - A°(n du / ov) du^2),
// the last entry (0, 0), so that a tap reads value + f * slope.
#include <math.h>

#include "psc_internal.cuh"

namespace psc {
namespace {

__device__ double aperture_value(int kind, double q, double dl, double alpha, const double *tab, int tab_len) {
    if (kind == PSC_AP_TABLE) {
        const double x = q / dl;
        if (!(x < 1.0)) return 0.0;
        const double t = x * (tab_len - 1);
        const int k = min((int)floor(t), tab_len - 2);
        const double f = t - k;
        return ((1.0 - f) * tab[k] + f * tab[k + 1]) / (dl * dl);
    }
    if (kind == PSC_AP_DISK) {
        if (q >= dl) return 0.0;
        const double R = 0.5 * dl;
        const double ovl = 2.0 * R * R * acos(q / (2.0 * R)) - 0.5 * q * sqrt(fmax(4.0 * R * R - q * q, 0.0));
        const double area = M_PI * R * R;
        return ovl / (area * area);
    }
    const double a2 = alpha * alpha;
    return (M_PI / (2.0 * a2)) * exp(-M_PI * M_PI * q * q / (2.0 * a2));
}

__global__ void tables_kernel(int kind, double diam_m, double alpha_per_dl, const double *ap_tab, int ap_len,
                              const double *freq, int nc, double du, int ov, const int *off, const int *len,
                              float2 *tabs) {
    const int c = blockIdx.y;
    if (c >= nc) return;
    const int n_len = len[c];
    const double dl = diam_m * freq[c] / kC;
    const double alpha = alpha_per_dl * dl;
    const double cell2 = du * du;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_len; n += gridDim.x * blockDim.x) {
        float2 e = make_float2(0.f, 0.f);
        if (n + 1 < n_len) {
            const double a0 = aperture_value(kind, n * du / ov, dl, alpha, ap_tab, ap_len) * cell2;
            const double a1 = aperture_value(kind, (n + 1) * du / ov, dl, alpha, ap_tab, ap_len) * cell2;
            e = make_float2((float)a0, (float)(a1 - a0));
        }
        tabs[off[c] + n] = e;
    }
}

}  // namespace

cudaError_t launch_tables(const psc_aperture &ap, const double *ap_table_dev, const double *freq_dev, int nc,
                          double du, int ov, int support, const int *tab_off_dev, const int *tab_len_dev,
                          float2 *tabs, cudaStream_t s) {
    (void)support;
    if (ap.kind == PSC_AP_TABLE && (!ap_table_dev || ap.table_len < 2)) return cudaErrorInvalidValue;
    dim3 grid(4, nc);
    tables_kernel<<<grid, 128, 0, s>>>(ap.kind, ap.diam_m, ap.alpha_per_dlambda, ap_table_dev, ap.table_len,
                                      freq_dev, nc, du, ov, tab_off_dev, tab_len_dev, tabs);
    return cudaGetLastError();
}

}  // namespace psc
