// Baseline coordinates from antenna positions (the observation geometry that
// Eq. ME's u, v, w come from): local horizon frame (east, north, up) at
// latitude phi to the equatorial frame, then to (u, v, w) of a source at
// hour angle H and declination delta; b_ij = x_j - x_i in metres, one row per
// baseline in the order (0,1), (0,2), ..., (1,2), ...  FP64 throughout.
#include <algorithm>

#include "psc_internal.cuh"

namespace psc {
namespace {

// One thread per (time, baseline).
__global__ void uvw_kernel(const double *__restrict__ enu, int n_ant, double sin_lat, double cos_lat, double sin_dec,
                           double cos_dec, const double *__restrict__ ha, int n_time, double *__restrict__ out) {
    const long long n_bl = (long long)n_ant * (n_ant - 1) / 2;
    const long long total = n_bl * n_time;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(k / n_bl);
        long long b = k - (long long)t * n_bl;
        // baseline b -> (i, j): row i holds n_ant - 1 - i pairs
        int i = 0;
        while (b >= n_ant - 1 - i) {
            b -= n_ant - 1 - i;
            ++i;
        }
        const int j = i + 1 + (int)b;
        const double de = enu[3 * j] - enu[3 * i];
        const double dn = enu[3 * j + 1] - enu[3 * i + 1];
        const double du = enu[3 * j + 2] - enu[3 * i + 2];
        const double X = -sin_lat * dn + cos_lat * du;
        const double Y = de;
        const double Z = cos_lat * dn + sin_lat * du;
        double sh, ch;
        sincos(ha[t], &sh, &ch);
        double *o = out + 3 * k;
        o[0] = sh * X + ch * Y;
        o[1] = -sin_dec * ch * X + sin_dec * sh * Y + cos_dec * Z;
        o[2] = cos_dec * ch * X - cos_dec * sh * Y + sin_dec * Z;
    }
}

}  // namespace

cudaError_t launch_uvw(const double *enu_dev, int n_ant, double lat, double dec, const double *ha_dev, int n_time,
                       double *uvw_dev, cudaStream_t s) {
    const long long total = (long long)n_ant * (n_ant - 1) / 2 * n_time;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 4096));
    uvw_kernel<<<blocks, 256, 0, s>>>(enu_dev, n_ant, sin(lat), cos(lat), sin(dec), cos(dec), ha_dev, n_time, uvw_dev);
    return cudaGetLastError();
}

}  // namespace psc
