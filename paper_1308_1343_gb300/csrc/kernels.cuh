// Device kernels of the level library (sm_103a, FP64).
//
// Traversal (the GPU form of the loop decomposition in arXiv 1308.1343,
// Sec. 3.1): the level's boxes are cut into work items (box, x-tile, y-tile,
// z-run).  A CTA takes items from a static stride over the item list (one
// persistent launch for all boxes of all domains).  Within an item, thread
// (lx, ly) owns the two x-adjacent points (x0 + 2 lx, x0 + 2 lx + 1) of row
// y0 + ly -- 16-byte loads and stores, rows 128-byte aligned by the level
// layout -- and marches up the z-run, keeping the five z-values k-2..k+2 of
// its column in registers.  The current plane of the tile plus a 2-point
// halo is staged in shared memory (double-buffered, one barrier per plane)
// for the in-plane neighbours.  Tile tails are handled by predication, as
// the paper's masked iteration does for vector tails (Sec. 4.3): points
// outside the box are loaded only where they are ghosts, and never stored.
//
// The Laplacian's 13-point integer-weighted sum has two arithmetic forms:
//  * Fp64:  FP64 adds and FMAs.
//  * Fixed: every input x is first rounded to the integer round(x * 2^S),
//    with S = 1077 - E and E the largest biased exponent of the field on
//    the box's domain, so |x| * 2^S < 2^55; the weighted sum (weights
//    16, -1, -90; sum of |weights| = 192 < 2^8) is then exact in int64 and
//    is rounded to FP64 once.  This moves the sum from GB300's narrow FP64
//    pipe to the integer pipes; only the RK updates stay FP64 FMAs.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "descriptors.hpp"

namespace sc {
namespace dev {

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double2 ld2(const double* p) {
  return *reinterpret_cast<const double2*>(p);
}
__device__ __forceinline__ void st2(double* p, double2 v) {
  *reinterpret_cast<double2*>(p) = v;
}
// Streaming load for data read once in this pass.
__device__ __forceinline__ double2 ld2_stream(const double* p) {
  return __ldcs(reinterpret_cast<const double2*>(p));
}

__device__ __forceinline__ unsigned biased_exp(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// round(x * 2^S) for |x| < 2^(E-1022), S = 1077 - E, without FP64
// instructions: unpack the significand and shift it into place (round half
// away from zero).  Zero and subnormal inputs give 0.  An input above the
// domain bound (shift > 2) is clamped and flagged.
__device__ __forceinline__ long long to_fix(double x, int S, unsigned& err) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = e + S - 1075;
  unsigned long long v;
  if (sh >= 0) {
    if (sh > 2) err |= kErrScale;
    v = m << (sh > 2 ? 2 : sh);
  } else {
    const int r = -sh;
    v = r >= 64 ? 0ull : (((m >> (r - 1)) + 1ull) >> 1);
  }
  if (e == 0) v = 0ull;
  const long long s = (long long)v;
  return (long long)(b >> 63) ? -s : s;
}

// ---------------------------------------------------------------------------
// Arithmetic policies for the 13-point sum
// ---------------------------------------------------------------------------

struct Fp64 {
  using T = double;
  using T2 = double2;
  static constexpr bool kFixed = false;
  int S = 0;  // unused
  // m0, m1: whether each value is one the stencil may read (unused here:
  // values outside the star are loaded but never used)
  __device__ __forceinline__ T2 conv(double2 v, bool, bool, unsigned&) const { return v; }
  __device__ __forceinline__ static T2 zero() { return make_double2(0.0, 0.0); }
  // r = 16 s1 - s2 - 90 c: the unscaled 12 h^2 L u
  __device__ __forceinline__ static T lap(T c, T xm1, T xp1, T ym1, T yp1, T zm1, T zp1,
                                          T xm2, T xp2, T ym2, T yp2, T zm2, T zp2) {
    const double s1 = ((xm1 + xp1) + (ym1 + yp1)) + (zm1 + zp1);
    const double s2 = ((xm2 + xp2) + (ym2 + yp2)) + (zm2 + zp2);
    return fma(-90.0, c, fma(16.0, s1, -s2));
  }
  __device__ __forceinline__ static double to_double(T r) { return r; }
};

struct Fixed {
  using T = long long;
  using T2 = longlong2;
  static constexpr bool kFixed = true;
  int S = 0;
  // Values outside the star of the box (edge and corner points of the padded
  // box, row padding) are never used; they are not converted, so whatever the
  // caller left there cannot raise the error word.
  __device__ __forceinline__ T2 conv(double2 v, bool m0, bool m1, unsigned& err) const {
    return make_longlong2(m0 ? to_fix(v.x, S, err) : 0ll, m1 ? to_fix(v.y, S, err) : 0ll);
  }
  __device__ __forceinline__ static T2 zero() { return make_longlong2(0, 0); }
  __device__ __forceinline__ static T lap(T c, T xm1, T xp1, T ym1, T yp1, T zm1, T zp1,
                                          T xm2, T xp2, T ym2, T yp2, T zm2, T zp2) {
    const long long s1 = ((xm1 + xp1) + (ym1 + yp1)) + (zm1 + zp1);
    const long long s2 = ((xm2 + xp2) + (ym2 + yp2)) + (zm2 + zp2);
    return s1 * 16 - s2 - c * 90;
  }
  __device__ __forceinline__ static double to_double(T r) { return __ll2double_rn(r); }
};

// ---------------------------------------------------------------------------
// The traversal
// ---------------------------------------------------------------------------

// Shared-memory tile: two buffers of (TX+4) x (TY+4) values, TX = 2*txh,
// TY = NT/txh, txh in {8, 16, 32, 64}; the extreme shapes bound the size.
template <int NT>
struct TileSmem {
  static constexpr int kA = (2 * 64 + 4) * (NT / 64 + 4);
  static constexpr int kB = (2 * 8 + 4) * (NT / 8 + 4);
  static constexpr int kMaxElems = kA > kB ? kA : kB;
};

// Walk one work item.  `F` is the stencil field (its ghosts filled).  For
// every plane k, epi.prefetch(idx) is called first (idx = element index of
// this thread's first point on plane k), then epi.point(idx, rA, rB, actA,
// actB) with the unscaled sums r = 12 h^2 (L F) at both points, converted to
// double.
template <int NT, class A, class Epi>
__device__ __forceinline__ void run_item(const DItem& it, const DBox& bx,
                                         const double* __restrict__ F, A arith,
                                         typename A::T* smem, unsigned& err, Epi& epi) {
  using T = typename A::T;
  using T2 = typename A::T2;
  const int txh = it.txh;
  const int TY = NT / txh;
  const int TX = 2 * txh;
  const int W = TX + 4;
  const int bufElems = W * (TY + 4);
  const int tid = threadIdx.x;
  const int lx = tid % txh, ly = tid / txh;
  const int gx = it.x0 + 2 * lx, gy = it.y0 + ly;
  const bool colLoad = (gx < bx.nx + 2) && (gy < bx.ny + 2);
  const bool actA = (gx < bx.nx) && (gy < bx.ny);
  const bool actB = (gx + 1 < bx.nx) && (gy < bx.ny);
  const long long colOff = bx.off + gx + (long long)gy * bx.py;
  const double* col = F + colOff;
  const long long pz = bx.pz;

  // a point is read by some stencil iff it lies outside the interior along
  // at most one axis, and there within the ghost width: out() is 0 inside,
  // 1 in the ghost range [-2, 0) or [n, n+2), 2 beyond (row padding)
  auto out = [](int c, int n) -> int {
    return (unsigned)c < (unsigned)n ? 0 : ((c >= -2 && c < n + 2) ? 1 : 2);
  };
  const int oy = out(gy, bx.ny);
  const int ox0 = out(gx, bx.nx), ox1 = out(gx + 1, bx.nx);
  auto ldcol = [&](int k) -> T2 {
    if (!colLoad) return A::zero();
    const int oz = out(k, bx.nz);
    return arith.conv(ld2(col + (long long)k * pz), ox0 + oy + oz <= 1, ox1 + oy + oz <= 1,
                      err);
  };

  T2 q0 = ldcol(it.z0 - 2), q1 = ldcol(it.z0 - 1), q2 = ldcol(it.z0), q3 = ldcol(it.z0 + 1);
  const int nhalo = 4 * txh + 2 * TY;
  const int rowSelf = (ly + 2) * W + 2 * lx + 2;

  for (int kk = 0; kk < it.nzr; ++kk) {
    const int k = it.z0 + kk;
    const T2 q4 = ldcol(k + 2);
    const long long idx = colOff + (long long)k * pz;
    if (actA) epi.prefetch(idx);
    T* buf = smem + (kk & 1) * bufElems;
    *reinterpret_cast<T2*>(buf + rowSelf) = q2;
    for (int h = tid; h < nhalo; h += NT) {
      int hx, hy;
      if (h < 4 * txh) {
        const int r = h / txh;
        hx = 2 * (h - r * txh);
        hy = r < 2 ? r - 2 : TY + r - 2;
      } else {
        const int j = h - 4 * txh;
        const int side = j / TY;
        hy = j - side * TY;
        hx = side ? TX : -2;
      }
      const int ax = it.x0 + hx, ay = it.y0 + hy;
      T2 v = A::zero();
      if (ax < bx.nx + 2 && ay < bx.ny + 2) {
        const int o = out(ay, bx.ny) + out(k, bx.nz);
        v = arith.conv(ld2(F + bx.off + ax + (long long)ay * bx.py + (long long)k * pz),
                       out(ax, bx.nx) + o <= 1, out(ax + 1, bx.nx) + o <= 1, err);
      }
      *reinterpret_cast<T2*>(buf + (hy + 2) * W + hx + 2) = v;
    }
    __syncthreads();
    if (actA) {
      const T* row = buf + rowSelf;
      const T2 xm = *reinterpret_cast<const T2*>(row - 2);
      const T2 xp = *reinterpret_cast<const T2*>(row + 2);
      const T2 ym1 = *reinterpret_cast<const T2*>(row - W);
      const T2 ym2 = *reinterpret_cast<const T2*>(row - 2 * W);
      const T2 yp1 = *reinterpret_cast<const T2*>(row + W);
      const T2 yp2 = *reinterpret_cast<const T2*>(row + 2 * W);
      // point A at x, point B at x+1
      const T rA = A::lap(q2.x, xm.y, q2.y, ym1.x, yp1.x, q1.x, q3.x,
                          xm.x, xp.x, ym2.x, yp2.x, q0.x, q4.x);
      const T rB = A::lap(q2.y, q2.x, xp.x, ym1.y, yp1.y, q1.y, q3.y,
                          xm.y, xp.y, ym2.y, yp2.y, q0.y, q4.y);
      epi.point(idx, A::to_double(rA), A::to_double(rB), actA, actB);
    }
    q0 = q1;
    q1 = q2;
    q2 = q3;
    q3 = q4;
  }
  __syncthreads();  // the next item reuses the buffers
}

// Largest biased exponent over the CTA, one atomicMax per CTA.
__device__ __forceinline__ void cta_max_to(unsigned v, unsigned* dst, unsigned* red) {
  v = __reduce_max_sync(0xffffffffu, v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned x = l < (int)(blockDim.x >> 5) ? red[l] : 0u;
    x = __reduce_max_sync(0xffffffffu, x);
    if (l == 0 && x) atomicMax(dst, x);
  }
  __syncthreads();
}

}  // namespace dev
}  // namespace sc
