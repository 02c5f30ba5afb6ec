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
// Latency hiding is a one-plane software pipeline: while plane k is
// computed, the pointwise fields of plane k+1 are in flight to shared memory
// by cp.async (no registers held), and so are the next raw column and halo
// values: to registers with one stencil field, by cp.async with several
// (where registers are the scarce resource).  Nothing loaded in an iteration
// is consumed in the same iteration.  With several stencil fields, two
// per-epilogue options reorder work without changing any result: a deferred
// epilogue (kDefer: plane k's pointwise work runs after plane k+1's
// conversions) and a halo split by (pair, field) over more warps
// (kHaloSplit).
//
// The Laplacian's 13-point integer-weighted sum has two arithmetic forms:
//  * Fp64:  FP64 adds and FMAs.
//  * Fixed: every input x is first turned into the integer
//    trunc(x * 2^S), S = 1077 - E, with E the largest biased exponent of
//    the field on the box's domain, so |x| * 2^S < 2^55; the weighted sum
//    (weights 16, -1, -90; sum of |weights| = 192 < 2^8) is then exact in
//    int64 and is rounded to FP64 once.  Each input is off by less than
//    2^-S <= 2^-54 * max|x|.  This moves the sum from GB300's narrow FP64
//    pipe to the integer pipes; the RK updates stay FP64 FMAs.
//
// Checked build (SC_BOUNDS_CHECK defined): the traversal verifies every
// element index it loads from or hands to an epilogue against the item's
// box (see run_items) and records a failure as kErrBounds in the error word
// instead of making the access.  Release builds compile the checks out.
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
// the same with the streaming (evict-first) cache hint
__device__ __forceinline__ void st2cs(double* p, double2 v) {
  __stcs(reinterpret_cast<double2*>(p), v);
}

__device__ __forceinline__ unsigned biased_exp(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// 16-byte asynchronous global -> shared copy (bypasses L1)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait until at most one committed group of this thread is still pending
__device__ __forceinline__ void cp_async_wait_one() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// wait until at most N committed groups of this thread are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait_n() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 64-bit logical right shift whose amount saturates: >= 64 gives 0.
__device__ __forceinline__ unsigned long long shr_sat(unsigned long long v, unsigned r) {
  unsigned long long d;
  asm("shr.b64 %0, %1, %2;" : "=l"(d) : "l"(v), "r"(r));
  return d;
}

// trunc(x * 2^S), S = 1077 - E, for |x| < 2^(E-1022), with integer
// instructions only and no branches: the significand, shifted left by 2, is
// shifted right by E - e (e the exponent of x), so an input with e == E
// lands just below 2^55.  Inputs with use == false (values the stencil never
// reads) get a shift of 64 and give 0; so do zero and subnormal inputs
// (e == 0, and E >= 64 is guaranteed by the caller).  An input above the
// domain bound (e > E) is clamped and flags kErrScale.
__device__ __forceinline__ long long to_fix(double x, int E, bool use, unsigned& err) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned long long m = ((b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 2;
  const int r = use ? E - e : 64;
  err |= r < 0 ? kErrScale : 0u;
  const long long v = (long long)shr_sat(m, (unsigned)max(r, 0));
  return (hi >> 31) ? -v : v;
}

// ---------------------------------------------------------------------------
// Ghost exchange fused into producers ("push")
// ---------------------------------------------------------------------------

// Push table of a level: per box, six groups of DPush entries -- axis d, and
// whether the sources lie in the low (side 0) or high (side 1) two-deep slab
// of the box; group g of box b spans entries [gofs[6b+g], gofs[6b+g+1]).
struct PushTab {
  const DPush* e;
  const int* gofs;
};

__device__ __forceinline__ void push_group(const PushTab& t, int g, int x, int y, int z, double v,
                                           double* f) {
  const int j1 = t.gofs[g + 1];
  for (int j = t.gofs[g]; j < j1; ++j) {
    const DPush p = t.e[j];
    if (x >= p.lo0 && x < p.hi0 && y >= p.lo1 && y < p.hi1 && z >= p.lo2 && z < p.hi2)
      f[p.dbase + (x - p.lo0) + (y - p.lo1) * p.dpy + (z - p.lo2) * p.dpz] = v;
  }
}

// Write v, the new value of interior point (x, y, z) of box b (extent n), to
// every ghost point that copies it.  Each ghost point has exactly one owner,
// so these writes never collide.
__device__ __forceinline__ void push_point(const PushTab& t, int b, int x, int y, int z, int nx,
                                           int ny, int nz, double v, double* f) {
  const int g = 6 * b;
  if (x < 2) push_group(t, g + 0, x, y, z, v, f);
  if (x >= nx - 2) push_group(t, g + 1, x, y, z, v, f);
  if (y < 2) push_group(t, g + 2, x, y, z, v, f);
  if (y >= ny - 2) push_group(t, g + 3, x, y, z, v, f);
  if (z < 2) push_group(t, g + 4, x, y, z, v, f);
  if (z >= nz - 2) push_group(t, g + 5, x, y, z, v, f);
}

// After a CTA has written work item `it` of field f (and passed a barrier),
// copy the item's points that other boxes read as ghosts: every push entry
// of the item's box is intersected with the item's region, and the CTA's
// threads copy the intersection.  Items away from all faces return at once.
template <int NT>
__device__ __forceinline__ void push_item(const PushTab& t, const DItem& it, const DBox& bx,
                                          double* f) {
  if (!t.gofs) return;  // no push table: the caller gathers instead
  const int xa = it.x0, xb = min(it.x0 + 2 * it.txh, bx.nx);
  const int ya = it.y0, yb = min(it.y0 + NT / it.txh, bx.ny);
  const int za = it.z0, zb = it.z0 + it.nzr;
  if (xa >= 2 && xb <= bx.nx - 2 && ya >= 2 && yb <= bx.ny - 2 && za >= 2 && zb <= bx.nz - 2)
    return;
  const int off0 = (int)bx.off, py = (int)bx.py, pz = (int)bx.pz;
  const int j0 = t.gofs[6 * it.box], j1 = t.gofs[6 * it.box + 6];
  for (int j = j0; j < j1; ++j) {
    const DPush p = t.e[j];
    const int lx = max(p.lo0, xa), hx = min(p.hi0, xb);
    const int ly = max(p.lo1, ya), hy = min(p.hi1, yb);
    const int lz = max(p.lo2, za), hz = min(p.hi2, zb);
    if (lx >= hx || ly >= hy || lz >= hz) continue;
    const int ex = hx - lx, ey = hy - ly, n = ex * ey * (hz - lz);
    for (int q = threadIdx.x; q < n; q += NT) {
      const int tq = q / ex;
      const int x = lx + (q - tq * ex);
      const int z = lz + tq / ey;
      const int y = ly + (tq - (z - lz) * ey);
      f[p.dbase + (x - p.lo0) + (y - p.lo1) * p.dpy + (z - p.lo2) * p.dpz] =
          f[off0 + x + y * py + z * pz];
    }
  }
}

// 2^k as a double for -1022 <= k <= 1023
__device__ __forceinline__ double exp2_int(int k) {
  return __longlong_as_double((long long)(1023 + k) << 52);
}

// ---------------------------------------------------------------------------
// Arithmetic policies for the 13-point sum
// ---------------------------------------------------------------------------

struct Fp64 {
  using T = double;
  using T2 = double2;
  static constexpr bool kFixed = false;
  int E = 0;  // unused
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
  // r * 2^(k - S) with S = 0: an exact power-of-two multiply
  __device__ __forceinline__ double scaled(T r, int k) const { return r * exp2_int(k); }
  // (r * 2^k0, r * 2^k1)
  __device__ __forceinline__ void scaled2(T r, int k0, int k1, double& d0, double& d1) const {
    d0 = r * exp2_int(k0);
    d1 = r * exp2_int(k1);
  }
};

struct Fixed {
  using T = long long;
  using T2 = longlong2;
  static constexpr bool kFixed = true;
  int E = 0;  // domain exponent bound of the stencil field
  // Values outside the star of the box (edge and corner points of the padded
  // box, row padding) are never used; they are not converted, so whatever the
  // caller left there cannot raise the error word.
  __device__ __forceinline__ T2 conv(double2 v, bool m0, bool m1, unsigned& err) const {
    return make_longlong2(to_fix(v.x, E, m0, err), to_fix(v.y, E, m1, err));
  }
  __device__ __forceinline__ static T2 zero() { return make_longlong2(0, 0); }
  __device__ __forceinline__ static T lap(T c, T xm1, T xp1, T ym1, T yp1, T zm1, T zp1,
                                          T xm2, T xp2, T ym2, T yp2, T zm2, T zp2) {
    const long long s1 = xm1 + xp1 + ym1 + yp1 + zm1 + zp1;
    const long long s2 = xm2 + xp2 + ym2 + yp2 + zm2 + zp2;
    return s1 * 16 - s2 - c * 90;
  }
  __device__ __forceinline__ static double to_double(T r) { return __ll2double_rn(r); }
  // r * 2^(k - S) rounded once: the conversion's exponent is adjusted on the
  // integer pipe (E >= 64 keeps it normal for every |r| >= 1).
  __device__ __forceinline__ double scaled(T r, int k) const {
    const long long bits = __double_as_longlong(__ll2double_rn(r)) +
                           ((long long)(k - (1077 - E)) << 52);
    return r == 0 ? 0.0 : __longlong_as_double(bits);
  }
  // scaled(r, k0) and scaled(r, k1) from one conversion (k0, k1 >= -8: a
  // nonzero result has |r| >= 1 and stays normal)
  __device__ __forceinline__ void scaled2(T r, int k0, int k1, double& d0, double& d1) const {
    const long long b = __double_as_longlong(__ll2double_rn(r)) - ((long long)(1077 - E) << 52);
    d0 = r == 0 ? 0.0 : __longlong_as_double(b + ((long long)k0 << 52));
    d1 = r == 0 ? 0.0 : __longlong_as_double(b + ((long long)k1 << 52));
  }
};

// The Fixed form with the int64 -> FP64 conversion on the integer pipes:
// the leading one is found with a count of leading zeros, the next 52 bits
// become the significand, rounded half away from zero on the 53rd (|error|
// <= 1/2 ulp; exact ties, which need the 53rd bit set and every lower bit
// clear, round away from zero instead of to even).  Used where FP64 issue
// slots, not integer ones, are the scarce resource: GB300 runs FP64 at two
// lanes per clock per SM, and the hardware conversion takes an FP64 slot.
struct FixedI : Fixed {
  // bits of r * 2^(k - S) less the k term, and whether r != 0
  __device__ __forceinline__ unsigned long long base_bits(T r, bool& nz) const {
    const unsigned long long a = r < 0 ? 0ull - (unsigned long long)r : (unsigned long long)r;
    const int lz = __clzll((long long)a);
    const unsigned long long m = a << (lz & 63);  // leading one at bit 63
    nz = a != 0;
    // (m >> 11) carries the leading one into the exponent field, hence 1085
    return (m >> 11) + ((m >> 10) & 1ull) +
           ((unsigned long long)(1085 - (1077 - E) - lz) << 52) +
           ((unsigned long long)r & 0x8000000000000000ull);
  }
  __device__ __forceinline__ double scaled(T r, int k) const {
    bool nz;
    const unsigned long long b = base_bits(r, nz) + ((unsigned long long)(long long)k << 52);
    return nz ? __longlong_as_double((long long)b) : 0.0;
  }
  __device__ __forceinline__ void scaled2(T r, int k0, int k1, double& d0, double& d1) const {
    bool nz;
    const unsigned long long b = base_bits(r, nz);
    d0 = nz ? __longlong_as_double((long long)(b + ((unsigned long long)(long long)k0 << 52))) : 0.0;
    d1 = nz ? __longlong_as_double((long long)(b + ((unsigned long long)(long long)k1 << 52))) : 0.0;
  }
};

// ---------------------------------------------------------------------------
// The traversal
// ---------------------------------------------------------------------------

// Shared memory of one CTA: two (TX+4) x (TY+4) stencil tiles, TX = 2*txh,
// TY = NT/txh, txh in {8, 16, 32} (the 64 x 8 tile bounds the size), and
// two planes of NF pointwise fields (one 16-byte pair per thread and field).
template <int NT>
struct TileSmem {
  static constexpr int kA = (2 * 32 + 4) * (NT / 32 + 4);
  static constexpr int kB = (2 * 8 + 4) * (NT / 8 + 4);
  static constexpr int kMaxElems = kA > kB ? kA : kB;
};

// NS stencil fields share the traversal (one pipeline, one barrier per
// plane); field f uses tile buffers 2f and 2f+1.  A deferred epilogue (see
// run_items) keeps three planes of pointwise fields instead of two.  ASYNC:
// the raw column and halo values are staged in shared memory by cp.async
// (the default with several stencil fields) instead of in registers.
template <int NT, class A, int NF, int NS = 1, bool DEFER = false, bool ASYNC = (NS > 1)>
struct Smem {
  typename A::T tile[2 * NS * TileSmem<NT>::kMaxElems];
  double2 pw[DEFER ? 3 : 2][NF > 0 ? NF : 1][NT];
  // raw halo pairs and raw column pairs staged by cp.async
  double2 hraw[2][NS][ASYNC ? NT : 1];
  double2 craw[2][NS][ASYNC ? NT : 1];
};

// Epi::kDefer if the epilogue declares it, else false
template <class E, class = void>
struct DeferOf {
  static constexpr bool value = false;
};
template <class E>
struct DeferOf<E, std::void_t<decltype(E::kDefer)>> {
  static constexpr bool value = E::kDefer;
};

// Epi::kHaloSplit if the epilogue declares it, else false
template <class E, class = void>
struct HaloSplitOf {
  static constexpr bool value = false;
};
template <class E>
struct HaloSplitOf<E, std::void_t<decltype(E::kHaloSplit)>> {
  static constexpr bool value = E::kHaloSplit;
};

// a point is read by some stencil iff it lies outside the interior along at
// most one axis, and there within the ghost width: 0 inside, 1 in the ghost
// range [-2, 0) or [n, n+2), 2 beyond (row padding)
__device__ __forceinline__ int out_of(int c, int n) {
  return (unsigned)c < (unsigned)n ? 0 : ((c >= -2 && c < n + 2) ? 1 : 2);
}

// Walk one work item over NS stencil fields F[0..NS) (ghosts filled), field
// f in the arithmetic arith[f].  The epilogue names Epi::NF pointwise fields
// (epi.f[0..NF)) that the traversal streams into shared memory; for every
// plane k it calls
//   epi.point(idx, pw, rA, rB, actB, x, y, k)
// on the threads owning interior points, with idx the element index of the
// thread's first point (x, y, k), pw[j] its pair of pointwise field j, and
// rA[f], rB[f] the unscaled sums r = 12 h^2 (L F[f]) at both points in the
// policy's integer or FP64 form.  With several stencil fields the epilogue
// may be deferred (Epi::kDefer): plane k's runs after plane k+1's
// conversions, before its barrier, which shortens the register lifetimes
// around the stencil; the arithmetic and its results are unchanged.
template <int NT, int NS, class A, class Epi, bool ASYNC = (NS > 1)>
__device__ __forceinline__ void run_items(
    const DItem& it, const DBox& bx, const double* const (&F)[NS], const A (&arith)[NS],
    Smem<NT, A, Epi::NF, NS, (NS > 1 && DeferOf<Epi>::value), ASYNC>& sm, unsigned& err,
    Epi& epi) {
  using T = typename A::T;
  using T2 = typename A::T2;
  constexpr int NF = Epi::NF;
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
  const int pz = (int)bx.pz;
  // in-plane coordinate c in [-2, n + 2) of a self-periodic box (bx.wrap):
  // its periodic image in [0, n), i.e. the owner of the ghost point;
  // otherwise c.  Computed once per item, outside the plane loop (the z
  // ghosts of such a box are still gathered: wrapping z would cost the
  // loop address arithmetic and registers)
  const bool wrap = bx.wrap != 0;
  auto wr = [wrap](int c, int n) { return !wrap ? c : (c < 0 ? c + n : (c >= n ? c - n : c)); };
  // element index of the thread's pair on plane 0 (32-bit: a field holds
  // fewer than 2^31 doubles); columns outside the padded box read the box's
  // interior corner instead (in bounds, masked off below, never used)
  const int off0 = (int)bx.off, py = (int)bx.py;
#ifdef SC_BOUNDS_CHECK
  // a 16-byte pair at element i must lie in the box's padded block (x from
  // -2 to the end of the row's padding, y and z from -2 to n+1); one that
  // does not is replaced by the interior corner and flagged
  const int blk0 = off0 - 2 - 2 * py - 2 * pz;
  const int blk1 = off0 - 3 + py + (bx.ny + 1) * py + (bx.nz + 1) * pz;
  auto ck = [&](int i) {
    if (i < blk0 || i + 1 > blk1) {
      err |= kErrBounds;
      return off0;
    }
    return i;
  };
  // the point(s) handed to the epilogue: interior, at the element index the
  // coordinates give; otherwise the call is skipped and flagged
  auto ok_pt = [&](int i, int x, int y, int z, bool two) {
    const bool ok = x >= 0 && x + (two ? 1 : 0) < bx.nx && y >= 0 && y < bx.ny && z >= 0 &&
                    z < bx.nz && i == off0 + x + y * py + z * pz;
    if (!ok) err |= kErrBounds;
    return ok;
  };
#else
  auto ck = [](int i) { return i; };
  auto ok_pt = [](int, int, int, int, bool) { return true; };
#endif
  const int colOff = colLoad ? off0 + wr(gx, bx.nx) + wr(gy, bx.ny) * py : off0;
  const int oy = out_of(gy, bx.ny);
  const int ox0 = out_of(gx, bx.nx) + oy, ox1 = out_of(gx + 1, bx.nx) + oy;

  // this thread's halo pair of the plane tile, if any (at most one: the
  // halo of a tile has 4 txh + 2 TY <= NT pairs for every allowed shape)
  const int nhalo = 4 * txh + 2 * TY;
  // With several stencil fields and Epi::kHaloSplit, when NS * nhalo <= NT,
  // each thread takes one (pair, field) entry instead of one pair of every
  // field: the halo conversions spread over NS times as many warps, which
  // shortens the slowest warp's way to the plane barrier (measured: faster
  // for the adjoint passes, slower for the forward ones).
  const bool hsplit = NS > 1 && HaloSplitOf<Epi>::value && NS * nhalo <= NT;
  const int hfield = hsplit ? tid / nhalo : 0;
  const int hp = hsplit ? tid - hfield * nhalo : tid;  // the thread's halo pair
  const bool hasH = hsplit ? tid < NS * nhalo : tid < nhalo;
  auto mine = [&](int f) { return hasH && (!hsplit || f == hfield); };
  int hs = 0;                 // smem index of the pair
  int hg = off0;              // element index of the pair on plane 0
  int hx0 = 2, hx1 = 2;       // outside counts (>= 2: masked off)
  if (hasH) {
    int hx, hy;
    if (hp < 4 * txh) {
      const int r = hp / txh;
      hx = 2 * (hp - r * txh);
      hy = r < 2 ? r - 2 : TY + r - 2;
    } else {
      const int j = hp - 4 * txh;
      const int side = j / TY;
      hy = j - side * TY;
      hx = side ? TX : -2;
    }
    const int ax = it.x0 + hx, ay = it.y0 + hy;
    hs = (hy + 2) * W + hx + 2;
    if (ax < bx.nx + 2 && ay < bx.ny + 2) {
      hg = off0 + wr(ax, bx.nx) + wr(ay, bx.ny) * py;
      const int o = out_of(ay, bx.ny);
      hx0 = out_of(ax, bx.nx) + o;
      hx1 = out_of(ax + 1, bx.nx) + o;
    }
  }
  auto conv_at = [&](int f, double2 raw, int k) -> T2 {
    const int oz = out_of(k, bx.nz);
    return arith[f].conv(raw, ox0 + oz <= 1, ox1 + oz <= 1, err);
  };

  // The raw halo pairs of plane k and column pairs of plane k+2 travel by
  // cp.async with the pointwise fields of plane k (ASYNC: the default with
  // several stencil fields, where registers are the scarce resource), or
  // are loaded to registers a plane ahead.
  constexpr bool kAsyncHalo = ASYNC;
  constexpr bool kDefer = kAsyncHalo && DeferOf<Epi>::value;

  // running element offsets (advance by one plane per iteration)
  int oc = colOff + (it.z0 + 2) * pz;                         // next column load
  int oh = hg + it.z0 * pz;                                   // next halo load
  int op = off0 + (colLoad ? gx + gy * py : 0) + it.z0 * pz;  // next pointwise stage
  int oi = op;                                                // current plane
  // buf: the halo/column buffer (plane parity); pbuf: the pointwise buffer
  auto stage_pw = [&](int buf, int pbuf) {
    if (actA) {
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async16(&sm.pw[pbuf][f][tid], epi.f[f] + ck(op));
    }
    if (kAsyncHalo) {
      const int t = kAsyncHalo ? tid : 0;
#pragma unroll
      for (int f = 0; f < NS; ++f)
        if (mine(f)) cp_async16(&sm.hraw[buf][f][t], F[f] + ck(oh));
#pragma unroll
      for (int f = 0; f < NS; ++f) cp_async16(&sm.craw[buf][f][t], F[f] + ck(oc));
      oh += pz;
      oc += pz;
    }
    cp_async_commit();
    op += pz;
  };

  T2 qa[NS], qb[NS], qc[NS], qd[NS], qe[NS];
  double2 rc[NS], rh[NS];  // raw column of plane k+2, raw halo pair of plane k
#pragma unroll
  for (int f = 0; f < NS; ++f) {
    qa[f] = conv_at(f, ld2(F[f] + ck(oc - 4 * pz)), it.z0 - 2);
    qb[f] = conv_at(f, ld2(F[f] + ck(oc - 3 * pz)), it.z0 - 1);
    qc[f] = conv_at(f, ld2(F[f] + ck(oc - 2 * pz)), it.z0);
    qd[f] = conv_at(f, ld2(F[f] + ck(oc - pz)), it.z0 + 1);
    if (!kAsyncHalo) {
      rc[f] = ld2(F[f] + ck(oc));
      rh[f] = ld2(F[f] + ck(oh));
    }
  }
  if (!kAsyncHalo) {
    oc += pz;
    oh += pz;
  }
  stage_pw(0, 0);
  // deferred epilogue: the pointwise buffer of the current plane (mod 3) and
  // the previous plane's sums
  int b3 = 0;
  typename A::T sA[NS], sB[NS];

  const int rowSelf = (ly + 2) * W + 2 * lx + 2;
  // one plane: m2..p1 hold planes k-2..k+1; p2 receives plane k+2
  auto plane = [&](int kk, const T2 (&m2)[NS], const T2 (&m1)[NS], const T2 (&c0)[NS],
                   const T2 (&p1)[NS], T2 (&p2)[NS]) {
    const int k = it.z0 + kk;
    const int oz = out_of(k, bx.nz);
#pragma unroll
    for (int f = 0; f < NS; ++f) {
      if (!kAsyncHalo) p2[f] = conv_at(f, rc[f], k + 2);
      T* buf = sm.tile + (2 * f + (kk & 1)) * bufElems;
      *reinterpret_cast<T2*>(buf + rowSelf) = c0[f];
      if (!kAsyncHalo && hasH)
        *reinterpret_cast<T2*>(buf + hs) =
            arith[f].conv(rh[f], hx0 + oz <= 1, hx1 + oz <= 1, err);
    }
    // issue the next plane's loads before waiting on this one
    if (kk + 1 < it.nzr) {
      if (!kAsyncHalo) {
#pragma unroll
        for (int f = 0; f < NS; ++f) {
          rc[f] = ld2(F[f] + ck(oc));
          rh[f] = ld2(F[f] + ck(oh));
        }
        oc += pz;
        oh += pz;
      }
      stage_pw((kk + 1) & 1, kDefer ? (b3 == 2 ? 0 : b3 + 1) : ((kk + 1) & 1));
    } else {
      cp_async_commit();
    }
    cp_async_wait_one();
    if (kAsyncHalo) {
      // this thread's own copies are complete and visible to it
      const int t = kAsyncHalo ? tid : 0;
#pragma unroll
      for (int f = 0; f < NS; ++f) {
        if (mine(f))
          *reinterpret_cast<T2*>(sm.tile + (2 * f + (kk & 1)) * bufElems + hs) =
              arith[f].conv(sm.hraw[kk & 1][f][t], hx0 + oz <= 1, hx1 + oz <= 1, err);
        p2[f] = conv_at(f, sm.craw[kk & 1][f][t], k + 2);
      }
    }
    if (kDefer && kk > 0 && actA && ok_pt(oi - pz, gx, gy, k - 1, actB)) {
      const int pb = b3 == 0 ? 2 : b3 - 1;
      double2 pw[NF > 0 ? NF : 1];
#pragma unroll
      for (int f = 0; f < NF; ++f) pw[f] = sm.pw[pb][f][tid];
      epi.point(oi - pz, pw, sA, sB, actB, gx, gy, k - 1);
    }
    __syncthreads();
    if (actA) {
      T rA[NS], rB[NS];
#pragma unroll
      for (int f = 0; f < NS; ++f) {
        const T* row = sm.tile + (2 * f + (kk & 1)) * bufElems + rowSelf;
        const T2 xm = *reinterpret_cast<const T2*>(row - 2);
        const T2 xp = *reinterpret_cast<const T2*>(row + 2);
        const T2 ym1 = *reinterpret_cast<const T2*>(row - W);
        const T2 ym2 = *reinterpret_cast<const T2*>(row - 2 * W);
        const T2 yp1 = *reinterpret_cast<const T2*>(row + W);
        const T2 yp2 = *reinterpret_cast<const T2*>(row + 2 * W);
        // point A at x, point B at x+1
        rA[f] = A::lap(c0[f].x, xm.y, c0[f].y, ym1.x, yp1.x, m1[f].x, p1[f].x,
                       xm.x, xp.x, ym2.x, yp2.x, m2[f].x, p2[f].x);
        rB[f] = A::lap(c0[f].y, c0[f].x, xp.x, ym1.y, yp1.y, m1[f].y, p1[f].y,
                       xm.y, xp.y, ym2.y, yp2.y, m2[f].y, p2[f].y);
      }
      if (kDefer) {
#pragma unroll
        for (int f = 0; f < NS; ++f) {
          sA[f] = rA[f];
          sB[f] = rB[f];
        }
      } else if (ok_pt(oi, gx, gy, k, actB)) {
        double2 pw[NF > 0 ? NF : 1];
#pragma unroll
        for (int f = 0; f < NF; ++f) pw[f] = sm.pw[kk & 1][f][tid];
        epi.point(oi, pw, rA, rB, actB, gx, gy, k);
      }
    }
    oi += pz;
    b3 = b3 == 2 ? 0 : b3 + 1;
  };
  // unrolled by the queue length so the five z-values never move
  for (int kk = 0;;) {
    plane(kk, qa, qb, qc, qd, qe);
    if (++kk >= it.nzr) break;
    plane(kk, qb, qc, qd, qe, qa);
    if (++kk >= it.nzr) break;
    plane(kk, qc, qd, qe, qa, qb);
    if (++kk >= it.nzr) break;
    plane(kk, qd, qe, qa, qb, qc);
    if (++kk >= it.nzr) break;
    plane(kk, qe, qa, qb, qc, qd);
    if (++kk >= it.nzr) break;
  }
  if (kDefer && actA && ok_pt(oi - pz, gx, gy, it.z0 + it.nzr - 1, actB)) {
    const int pb = b3 == 0 ? 2 : b3 - 1;
    double2 pw[NF > 0 ? NF : 1];
#pragma unroll
    for (int f = 0; f < NF; ++f) pw[f] = sm.pw[pb][f][tid];
    epi.point(oi - pz, pw, sA, sB, actB, gx, gy, it.z0 + it.nzr - 1);
  }
  cp_async_wait_all();
  __syncthreads();  // the next item reuses the buffers
}

// One stencil field: epi.point receives the two sums as scalars.
template <class Epi>
struct OneField {
  static constexpr int NF = Epi::NF;
  Epi& e;
  const double* const* f;
  template <class T>
  __device__ __forceinline__ void point(int i, const double2* pw, const T (&rA)[1],
                                        const T (&rB)[1], bool actB, int x, int y, int k) {
    e.point(i, pw, rA[0], rB[0], actB, x, y, k);
  }
};

template <int NT, class A, class Epi, bool ASYNC = false>
__device__ __forceinline__ void run_item(const DItem& it, const DBox& bx,
                                         const double* __restrict__ F, A arith,
                                         Smem<NT, A, Epi::NF, 1, false, ASYNC>& sm,
                                         unsigned& err, Epi& epi) {
  const double* const Fs[1] = {F};
  const A as[1] = {arith};
  OneField<Epi> one{epi, epi.f};
  run_items<NT, 1, A, OneField<Epi>, ASYNC>(it, bx, Fs, as, sm, err, one);
}

// Largest biased exponents of two fields over the CTA, one atomicMax per CTA
// and field (red holds 2 * warps entries).
__device__ __forceinline__ void cta_max2_to(unsigned a, unsigned b, unsigned* da, unsigned* db,
                                            unsigned* red) {
  a = __reduce_max_sync(0xffffffffu, a);
  b = __reduce_max_sync(0xffffffffu, b);
  const int nw = (int)(blockDim.x >> 5);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[w] = a;
    red[nw + w] = b;
  }
  __syncthreads();
  if (w == 0) {
    unsigned x = l < nw ? red[l] : 0u, y = l < nw ? red[nw + l] : 0u;
    x = __reduce_max_sync(0xffffffffu, x);
    y = __reduce_max_sync(0xffffffffu, y);
    if (l == 0) {
      if (x) atomicMax(da, x);
      if (y) atomicMax(db, y);
    }
  }
  __syncthreads();
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
