// HEALPix pixel centres for the library (host only, compiled with
// -ffp-contract=off).  The paper emits N_rays = 12 * 4^l HEALPix rays per
// source (Sec. 2); the centres follow the ring equations of Gorski et al.
// 2005 in RING order.  Each pixel index is mapped to its ring and position,
// then evaluated with a fixed sequence of IEEE operations:
//   z     = zn / zd                      (integers zn, zd)
//   sin t = sqrt(zd^2 - zn^2) / zd
//   phi   = (pi/2) * (k + r/den), k the quadrant; cos and sin of the in-quadrant
//           angle come from the first octant (swapping cos and sin above pi/4,
//           both sqrt(1/2) at pi/4), so mirror-symmetric pixels have
//           bitwise-equal component magnitudes;
//   m     = (sin t cos phi, sin t sin phi, z), negative zeros made positive.
#include <math.h>
#include <stdint.h>

#include "../../include/rt_api.h"

namespace {

// ring (1-based, north to south) and position in ring (1-based) of pixel p
void ring_of_pixel(int64_t N, int64_t p, int64_t* ring, int64_t* pos)
{
    const int64_t ncap = 2 * N * (N - 1);
    const int64_t npix = 12 * N * N;
    if (p < ncap) {
        int64_t i = (int64_t)((1.0 + sqrt(1.0 + 2.0 * (double)p)) * 0.5);
        while (i > 1 && 2 * i * (i - 1) > p) i--;  // ring i starts at pixel 2 i (i - 1)
        while (2 * (i + 1) * i <= p) i++;
        *ring = i;
        *pos = p - 2 * i * (i - 1) + 1;
    } else if (p < npix - ncap) {
        const int64_t q = p - ncap;
        *ring = N + q / (4 * N);
        *pos = q % (4 * N) + 1;
    } else {
        const int64_t pp = npix - 1 - p;  // counted back from the south pole
        int64_t i = (int64_t)((1.0 + sqrt(1.0 + 2.0 * (double)pp)) * 0.5);
        while (i > 1 && 2 * i * (i - 1) > pp) i--;
        while (2 * (i + 1) * i <= pp) i++;
        *ring = 4 * N - i;
        *pos = 4 * i - (pp - 2 * i * (i - 1));
    }
}

void quarter_turn_cos_sin(int64_t r, int64_t den, double* c, double* s)
{
    if (2 * r == den) {
        const double h = sqrt(0.5);
        *c = h;
        *s = h;
        return;
    }
    const bool upper = 2 * r > den;
    const int64_t rr = upper ? den - r : r;
    const double a = (M_PI / 2.0) * (double)rr / (double)den;
    const double ca = cos(a), sa = sin(a);
    *c = upper ? sa : ca;
    *s = upper ? ca : sa;
}

}  // namespace

extern "C" int rt_healpix_dirs(int nside, double* h_out)
{
    if (nside < 1 || nside > 1024 || (nside & (nside - 1)) || !h_out) return RT_ERR_ARG;
    const int64_t N = nside;
    for (int64_t p = 0; p < 12 * N * N; p++) {
        int64_t i, j;
        ring_of_pixel(N, p, &i, &j);
        int64_t zn, zd, num, den;
        if (i < N || i > 3 * N) {
            const int64_t ii = i < N ? i : 4 * N - i;
            zd = 3 * N * N;
            zn = zd - ii * ii;
            if (i > 3 * N) zn = -zn;
            num = 2 * j - 1;
            den = 2 * ii;
        } else {
            zd = 3 * N;
            zn = 4 * N - 2 * i;
            num = 2 * (j - 1) + (((i - N) & 1) == 0 ? 1 : 0);
            den = 2 * N;
        }
        double c, s;
        quarter_turn_cos_sin(num % den, den, &c, &s);
        double cphi, sphi;
        switch (num / den) {
        case 0: cphi = c; sphi = s; break;
        case 1: cphi = -s; sphi = c; break;
        case 2: cphi = -c; sphi = -s; break;
        default: cphi = s; sphi = -c; break;
        }
        const double st = sqrt((double)(zd * zd - zn * zn)) / (double)zd;
        double* v = h_out + 3 * p;
        v[0] = st * cphi;
        v[1] = st * sphi;
        v[2] = (double)zn / (double)zd;
        for (int b = 0; b < 3; b++)
            if (v[b] == 0.0) v[b] = 0.0;
    }
    return RT_OK;
}
