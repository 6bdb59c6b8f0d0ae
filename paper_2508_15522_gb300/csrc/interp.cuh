// Device helpers of the grid interpolation shared by the kernels of the
// relaxation / dynamics path and of the point-evaluation path: the cubic
// B-spline basis weights (Eq. Bspline) and the fold into the periodic tile
// with the cell index and fractional coordinates (Sec. 4, Sec. 5).
#pragma once

#include "internal.h"

namespace {

// Cubic B-spline weights w_j = B(t - j), j = -1..2, and dB/dt for t in [0,1),
// the polynomial pieces of Eq. Bspline on the four intervals.
__device__ __forceinline__ void bspline_weights(float t, float w[4], float dw[4]) {
  const float s = 1.f - t, t2 = t * t, t3 = t2 * t;
  const float sixth = 1.f / 6.f;
  w[0] = s * s * s * sixth;
  w[1] = fmaf(3.f, t3, fmaf(-6.f, t2, 4.f)) * sixth;
  w[2] = fmaf(-3.f, t3, fmaf(3.f, t2, fmaf(3.f, t, 1.f))) * sixth;
  w[3] = t3 * sixth;
  dw[0] = -0.5f * s * s;
  dw[1] = fmaf(1.5f, t2, -2.f * t);
  dw[2] = fmaf(-1.5f, t2, t + 0.5f);
  dw[3] = 0.5f * t2;
}

// Fold into the periodic tile (Sec. 4), cell index and fractional
// coordinates of one atom.
struct Cell {
  int ix, iy, iz;
  float tx, ty, tz;
  bool inside;   // inside the grid's z range (else the field is ~0)
};

__device__ __forceinline__ Cell locate(const GridView& g, bool act, float x, float y, float z, int& flags) {
  Cell c;
  float xr = x - g.x0, yr = y - g.y0;
  xr = fmaf(-g.Lx, floorf(xr * g.inv_Lx), xr);
  yr = fmaf(-g.Ly, floorf(yr * g.inv_Ly), yr);
  float ux = xr * g.inv_dx, uy = yr * g.inv_dy, uz = (z - g.z0) * g.inv_dz;
  float flx = floorf(ux), fly = floorf(uy);
  c.tx = fminf(fmaxf(ux - flx, 0.f), 1.f);
  c.ty = fminf(fmaxf(uy - fly, 0.f), 1.f);
  int ix = (int)flx, iy = (int)fly;
  if (ix >= g.nx) ix -= g.nx;
  if (iy >= g.ny) iy -= g.ny;
  c.ix = min(max(ix, 0), g.nx - 1);     // any input, even non-finite, stays in bounds
  c.iy = min(max(iy, 0), g.ny - 1);
  if (act && uz < g.uzf) flags |= GRIDFF_REP_BELOW;   // below the floor (ghost planes or lower)
  uz = fmaxf(uz, 0.f);
  c.inside = act && (uz < (float)(g.nz - 1));   // above the grid (or NaN): field ~ 0
  float flz = floorf(c.inside ? uz : 0.f);
  c.tz = (c.inside ? uz : 0.f) - flz;
  c.iz = min(max((int)flz, 0), g.nz - 2);
  return c;
}

}  // namespace
