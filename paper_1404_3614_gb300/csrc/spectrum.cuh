// Closed-form Fourier coefficients of the matrix-inclusion coefficient, evaluated from
// per-axis phase and sinc tables (Lemma bounds_for_matrix-inclusion, Remark "inclusion";
// ball and disk transforms of the indicator).
#pragma once
#include <math.h>

#include "kernels.cuh"

namespace homb {

// (sin q - q cos q) / q^3, with its Taylor series near 0
__device__ __forceinline__ double ball_radial(double q) {
  if (q < 0.1) {
    const double q2 = q * q;
    return 1.0 / 3.0 + q2 * (-1.0 / 30.0 + q2 * (1.0 / 840.0 + q2 * (-1.0 / 45360.0 + q2 / 3991680.0)));
  }
  double s, c;
  sincos(q, &s, &c);
  return (s - q * c) / (q * q * q);
}

// J1(q) / q, with its Taylor series near 0
__device__ __forceinline__ double disk_radial(double q) {
  if (q < 1e-3) return 0.5 - q * q / 16.0;
  return j1(q) / q;
}

// Radial factor 4 pi R^3 (sin q - q cos q)/q^3 (ball) or 2 pi R^2 J1(q)/q (disk), q = 2 pi R |xi|
__device__ __forceinline__ double radial_factor(int d, double R, double xi_norm) {
  const double q = 2.0 * M_PI * R * xi_norm;
  return d == 3 ? 4.0 * M_PI * R * R * R * ball_radial(q) : 2.0 * M_PI * R * R * disk_radial(q);
}

__device__ __forceinline__ void ahat_eval(const SpecArgs& a, const int* ni, const int* ns, double2* out) {
  for (int q = 0; q < a.ncomp; ++q) out[q] = make_double2(0.0, 0.0);
  if (ns[0] == 0 && ns[1] == 0 && ns[2] == 0)
    for (int q = 0; q < a.ncomp; ++q) out[q].x = a.A0p[q];
  double rad = 0.0;
  int grp = -1;
  const int n2 = ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2];
  for (int j = 0; j < a.nincl; ++j) {
    const DevIncl& I = a.incl[j];
    double f;
    if (I.shape == 0) {
      f = a.invVol;
      for (int al = 0; al < a.d; ++al) f *= a.sinc[((long long)j * 3 + al) * a.Mmax + ni[al]];
    } else {
      if (!I.same_as_prev) {
        ++grp;
        if (a.radtab) {
          rad = a.radtab[(long long)grp * a.radlen + n2];
        } else {
          double xi2 = 0.0;
          for (int al = 0; al < a.d; ++al) {
            const double xi = ns[al] * a.invY[al];
            xi2 += xi * xi;
          }
          rad = radial_factor(a.d, I.h[0], sqrt(xi2));
        }
      }
      f = rad * a.invVol;
    }
    double2 ph = a.phase[((long long)j * 3 + 0) * a.Mmax + ni[0]];
    for (int al = 1; al < a.d; ++al) {
      const double2 t = a.phase[((long long)j * 3 + al) * a.Mmax + ni[al]];
      ph = make_double2(ph.x * t.x - ph.y * t.y, ph.x * t.y + ph.y * t.x);
    }
    for (int q = 0; q < a.ncomp; ++q) {
      const double s = f * I.dA[q];
      out[q].x = fma(s, ph.x, out[q].x);
      out[q].y = fma(s, ph.y, out[q].y);
    }
  }
}


__device__ __forceinline__ int sym_index(int d, int al, int be) {
  if (al == be) return al;
  const int lo = al < be ? al : be, hi = al < be ? be : al;
  if (d == 2) return 2;
  if (lo == 1 && hi == 2) return 3;
  if (lo == 0 && hi == 2) return 4;
  return 5;
}


}  // namespace homb
