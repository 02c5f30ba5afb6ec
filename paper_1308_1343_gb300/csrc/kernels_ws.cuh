// Warp-specialised traversal of the two-stage pass kernels (sm_103a).
//
// The one-role traversal (run_items in kernels.cuh) keeps every warp of a CTA
// in the same phase -- one barrier per plane -- so the integer work of the
// fixed-point sums and the FP64 work of the RK epilogue of one CTA do not run
// at the same time, and the registers of both bound the warps per SM.  Here a
// CTA of 384 threads splits the work of each plane between two roles:
//
//  * 8 producer warps (256 threads) own the tile as before: thread (lx, ly)
//    holds the two x-adjacent points of its column, keeps the five z-values of
//    both stencil fields in registers, stages the raw column and halo values
//    of the coming planes by cp.async, converts them and forms the two 13-term
//    sums of both fields.  They synchronise among themselves once per plane
//    (the in-plane neighbours live in shared memory) and write the sums of
//    each plane to a ring of shared-memory slots;
//  * 4 consumer warps (128 threads, two point pairs each) take the sums of a
//    plane from the ring, stream the pointwise fields of their pairs by
//    cp.async one plane ahead, and run the epilogue (the int64 -> FP64
//    conversion of the sums, the FP64 FMAs, the stores, the exponent bounds).
//
// Producers and consumers hand over through mbarriers ("full" slot: the
// producers' 256 arrivals; "empty" slot: the consumers' 128 arrivals), so the
// two roles drift by up to kWsRing planes and the FP64 pipe runs beside the
// integer pipes.  The arithmetic of every point is that of run_items with the
// same epilogue: results are bit-identical to the one-role kernels.
//
// Every wait is bounded: a wait that has not seen its phase complete within
// kWsWaitNs (1 s) gives up, sets the CTA's abort flag and returns false; the
// other threads of the CTA see the flag in their own waits and return as
// well, and the kernel records kErrTimeout in the device error word, which
// sc_level_sync reports as SC_EDEVICE.  There are no named barriers after the
// start, so a thread that gives up cannot leave others blocked.
#pragma once

#include "kernels.cuh"

namespace sc {
namespace dev {

constexpr int kWsProducers = 256;  // 8 warps
#ifndef SC_WS_CONSUMERS
#define SC_WS_CONSUMERS 128
#endif
constexpr int kWsConsumers = SC_WS_CONSUMERS;  // 4 warps: one per SM sub-partition
constexpr int kWsThreads = kWsProducers + kWsConsumers;
constexpr int kWsPairs = kWsProducers / kWsConsumers;  // point pairs per consumer thread
constexpr int kWsRing = 2;  // sum slots: producers run at most 2 planes ahead
constexpr unsigned long long kWsWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// arrive (release semantics: this thread's earlier shared-memory writes are
// visible to a thread whose wait on the phase succeeds)
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

// true once the phase of parity `parity` has completed (acquire semantics);
// the thread may sleep up to kWsSuspendNs waiting for it instead of spinning
constexpr unsigned kWsSuspendNs = 1000000u;
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kWsSuspendNs)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of parity `parity`: false if kWsWaitNs pass
// first or another thread of the CTA has given up (*abort != 0).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort != 0 || global_ns() - t0 > kWsWaitNs) return false;
  }
}

// Shared memory of one warp-specialised CTA with two stencil fields and NF
// pointwise fields staged NB planes deep (NB = 2: one plane ahead; NB = 1:
// each pair's next plane as soon as its values are read): 107 KB for the
// forward passes (NF = 4, NB = 2), two CTAs per SM.
template <class A, int NF = 4, int NB = 2>
struct WsSmem {
  using Arith = A;
  static constexpr int kNF = NF;
  static constexpr int kNB = NB;
  typename A::T tile[2 * 2 * TileSmem<kWsProducers>::kMaxElems];  // [field][plane parity]
  double2 hraw[2][2][kWsProducers];   // [plane parity][field][producer]
  double2 craw[2][2][kWsProducers];
  typename A::T2 ring[kWsRing][2][kWsProducers];  // sums at (point A, point B)
  double2 pw[NB][NF][kWsProducers];   // [plane parity][field][pair]
  unsigned long long full[kWsRing];
  unsigned long long empty[kWsRing];
  unsigned long long tbar;            // producers: plane tile complete
  int abort;
};

// Register budgets of the two roles (setmaxnreg): the CTA is launched with
// kWsLaunchRegs per thread (two CTAs per SM: 80 for 384 threads), the
// producers take P and the consumers give back to what is left of the CTA's
// registers (P = 96: 48; P = 88: 64), rounded down to a multiple of 8.
constexpr int kWsLaunchRegs = 65536 / (2 * kWsThreads) / 8 * 8;
template <int P>
struct WsBudget {
  static constexpr int kConsumer =
      (kWsThreads * kWsLaunchRegs - kWsProducers * P) / kWsConsumers / 8 * 8;
  static_assert(kConsumer >= 24 && P <= 256, "register split");
};
template <int P>
__device__ __forceinline__ void ws_producer_regs() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(P) : "memory");
}
template <int P>
__device__ __forceinline__ void ws_consumer_regs() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(WsBudget<P>::kConsumer) : "memory");
}

// x-face ghost copies read from their owners (DXGhost): per box b, entries
// [ofs[2 b + side], ofs[2 b + side + 1]) of its low (side 0) and high (side
// 1) x face; ofs == NULL: none (every ghost the kernels read is gathered)
struct XgTab {
  const DXGhost* e;
  const int* ofs;
  const DBox* boxes;
};

// The copy that holds ghost row y of planes [z, z + n) of face g (2 b +
// side), or NULL (the row is gathered; work items at an x face end their
// z-run where such a copy starts or ends, so no item has a row in two)
__device__ __forceinline__ const DXGhost* xg_find(const XgTab& t, int g, int y, int z, int n) {
  for (int j = t.ofs[g], j1 = t.ofs[g + 1]; j < j1; ++j) {
    const DXGhost* e = t.e + j;
    if (y >= e->y0 && y < e->y1 && z >= e->z0 && z + n <= e->z1) return e;
  }
  return nullptr;
}

template <class S>
__device__ __forceinline__ void ws_init(S& sm) {
  if (threadIdx.x == 0) {
    for (int r = 0; r < kWsRing; ++r) {
      mbar_init(&sm.full[r], kWsProducers);
      mbar_init(&sm.empty[r], kWsConsumers);
    }
    mbar_init(&sm.tbar, kWsProducers);
    sm.abort = 0;
  }
  __syncthreads();
}

// Producer role for one work item (threads 0..255).  g counts the planes the
// CTA has handed over since the launch (ring slot and barrier phases follow
// it).  Returns false if a wait gave up.
template <class A, class S>
__device__ __forceinline__ bool ws_produce(const DItem& it, const DBox& bx,
                                           const double* const (&F)[2], const A (&arith)[2],
                                           S& sm, unsigned& err, unsigned& g,
                                           const XgTab& xt) {
  using T = typename A::T;
  using T2 = typename A::T2;
  const int txh = it.txh;
  const int TY = kWsProducers / txh;
  const int TX = 2 * txh;
  const int W = TX + 4;
  // buffers of (field, plane parity) at a fixed stride, whatever the item's
  // tile shape: a fast producer starting the next item writes the other
  // parity than the one slower producers may still be reading (there is no
  // CTA-wide barrier between items)
  constexpr int bufElems = TileSmem<kWsProducers>::kMaxElems;
  const int tid = threadIdx.x;
  const int lx = tid % txh, ly = tid / txh;
  const int gx = it.x0 + 2 * lx, gy = it.y0 + ly;
  const bool colLoad = (gx < bx.nx + 2) && (gy < bx.ny + 2);
  const bool actA = (gx < bx.nx) && (gy < bx.ny);
  const int pz = (int)bx.pz;
  const bool wrap = bx.wrap != 0;
  auto wr = [wrap](int c, int n) { return !wrap ? c : (c < 0 ? c + n : (c >= n ? c - n : c)); };
  const int off0 = (int)bx.off, py = (int)bx.py;
#ifdef SC_BOUNDS_CHECK
  const int blk0 = off0 - 2 - 2 * py - 2 * pz;
  const int blk1 = off0 - 3 + py + (bx.ny + 1) * py + (bx.nz + 1) * pz;
  auto ck = [&](int i) {
    if (i < blk0 || i + 1 > blk1) {
      err |= kErrBounds;
      return off0;
    }
    return i;
  };
#else
  auto ck = [](int i) { return i; };
#endif
  // Column and halo pairs are read at a plane-0 offset + k * pitch.  A pair
  // in the x-face ghosts of a box with neighbours (gx or ax is -2 or nx, its
  // row inside the box) is read from the box that owns it where the table
  // holds its copy: the owner's offset and plane pitch.  The item's planes
  // lie in that one copy (work items end their z-run where the owner
  // changes); the column's two planes beyond on either side are not used and
  // lie in the owner's padded block.
  const bool xgt = xt.ofs != nullptr && !wrap;
  int colOff = colLoad ? off0 + wr(gx, bx.nx) + wr(gy, bx.ny) * py : off0;
  int cpz = pz, hpz = pz;
  bool cN = false, hN = false;  // the column / halo pair reads another box
  // the owner of ghost row y of face fg (2 box + side) over the item's
  // planes: offset and pitch, or false (the row is gathered)
  auto owner = [&](int fg, int y, int& off, int& pitch) -> bool {
    const DXGhost* e = xg_find(xt, fg, y, it.z0, it.nzr);
    if (!e) return false;
    const int o = e->src + (y - e->y0) * e->spy - e->z0 * e->spz;
#ifdef SC_BOUNDS_CHECK
    const DBox& sb = xt.boxes[e->sbox];
    const int s0 = (int)sb.off - 2 - 2 * (int)sb.py - 2 * (int)sb.pz;
    const int s1 = (int)sb.off - 3 + (int)sb.py + (sb.ny + 1) * (int)sb.py + (sb.nz + 1) * (int)sb.pz;
    if (o + (it.z0 - 2) * e->spz < s0 || o + (it.z0 + it.nzr + 1) * e->spz + 1 > s1) {
      err |= kErrBounds;
      return false;
    }
#endif
    off = o;
    pitch = e->spz;
    return true;
  };
  if (xgt && colLoad && gx == bx.nx && gy < bx.ny) cN = owner(2 * it.box + 1, gy, colOff, cpz);
  const int oy = out_of(gy, bx.ny);
  const int ox0 = out_of(gx, bx.nx) + oy, ox1 = out_of(gx + 1, bx.nx) + oy;
  // this thread's halo pair of the plane tile, if any (at most one: the halo
  // of a tile has 4 txh + 2 TY <= 256 pairs for every allowed shape): rows
  // -2, -1, TY, TY+1 of the tile's columns, then columns -2 and TX of its rows
  const int nhalo = 4 * txh + 2 * TY;
  const bool hasH = tid < nhalo;
  int hs = 0, hg = off0, hx0 = 2, hx1 = 2;
  if (hasH) {
    int hx, hy;
    if (tid < 4 * txh) {
      const int r = tid / txh;
      hx = 2 * (tid - r * txh);
      hy = r < 2 ? r - 2 : TY + r - 2;
    } else {
      const int j = tid - 4 * txh;
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
      // (a pair of the rows above or below the tile is one too where the
      // tile is ragged in x)
      if (xgt && (ax == -2 || ax == bx.nx) && ay >= 0 && ay < bx.ny)
        hN = owner(2 * it.box + (ax < 0 ? 0 : 1), ay, hg, hpz);
    }
  }
#ifdef SC_BOUNDS_CHECK
  auto ckc = [&](int i) { return cN ? i : ck(i); };
  auto ckh = [&](int i) { return hN ? i : ck(i); };
#else
  auto ckc = ck;
  auto ckh = ck;
#endif
  auto conv_at = [&](int f, double2 raw, int k) -> T2 {
    const int oz = out_of(k, bx.nz);
    return arith[f].conv(raw, ox0 + oz <= 1, ox1 + oz <= 1, err);
  };
  // a self-periodic box of at least two planes (bx.wrap & 2) reads its z
  // ghosts from their periodic images too -- planes -2, -1 are nz-2, nz-1 and
  // planes nz, nz+1 are 0, 1 -- so that it needs no gather at all: the column
  // pointer goes back to plane 0 after plane nz-1 (halo loads stay inside)
  const bool zwrap = (bx.wrap & 2) != 0;
  auto wz = [&](int k) {
    return !zwrap ? k : (k < 0 ? k + bx.nz : (k >= bx.nz ? k - bx.nz : k));
  };
  const int ocLast = zwrap ? colOff + (bx.nz - 1) * pz : -1;
  int oc = colOff + wz(it.z0 + 2) * cpz;  // next column load (plane k+2)
  int oh = hg + it.z0 * hpz;              // next halo load (plane k)
  // raw halo pairs of plane k and column pairs of plane k+2, by cp.async
  auto stage_raw = [&](int buf) {
#pragma unroll
    for (int f = 0; f < 2; ++f)
      if (hasH) cp_async16(&sm.hraw[buf][f][tid], F[f] + ckh(oh));
#pragma unroll
    for (int f = 0; f < 2; ++f) cp_async16(&sm.craw[buf][f][tid], F[f] + ckc(oc));
    oh += hpz;
    oc = oc == ocLast ? colOff : oc + cpz;
    cp_async_commit();
  };
  T2 qa[2], qb[2], qc[2], qd[2], qe[2];
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    qa[f] = conv_at(f, ld2(F[f] + ckc(colOff + wz(it.z0 - 2) * cpz)), it.z0 - 2);
    qb[f] = conv_at(f, ld2(F[f] + ckc(colOff + wz(it.z0 - 1) * cpz)), it.z0 - 1);
    qc[f] = conv_at(f, ld2(F[f] + ckc(colOff + it.z0 * cpz)), it.z0);
    qd[f] = conv_at(f, ld2(F[f] + ckc(colOff + wz(it.z0 + 1) * cpz)), it.z0 + 1);
  }
  stage_raw(g & 1);
  const int rowSelf = (ly + 2) * W + 2 * lx + 2;
  // one plane: m2..p1 hold planes k-2..k+1; p2 receives plane k+2
  auto plane = [&](int kk, const T2 (&m2)[2], const T2 (&m1)[2], const T2 (&c0)[2],
                   const T2 (&p1)[2], T2 (&p2)[2]) -> bool {
    const int k = it.z0 + kk;
    const int oz = out_of(k, bx.nz);
    const int tb = (int)(g & 1u);
#pragma unroll
    for (int f = 0; f < 2; ++f)
      *reinterpret_cast<T2*>(sm.tile + (2 * f + tb) * bufElems + rowSelf) = c0[f];
    if (kk + 1 < it.nzr)
      stage_raw(tb ^ 1);
    else
      cp_async_commit();
    cp_async_wait_one();  // this thread's raw values of plane k have landed
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      if (hasH)
        *reinterpret_cast<T2*>(sm.tile + (2 * f + tb) * bufElems + hs) =
            arith[f].conv(sm.hraw[tb][f][tid], hx0 + oz <= 1, hx1 + oz <= 1, err);
      p2[f] = conv_at(f, sm.craw[tb][f][tid], k + 2);
    }
    // every producer has written plane k's tile
    mbar_arrive(&sm.tbar);
    if (!mbar_wait(&sm.tbar, g & 1u, &sm.abort)) return false;
    // the slot is free once the consumers released it; each field's sums go
    // to it as soon as they are formed
    const unsigned slot = g % kWsRing;
    if (!mbar_wait(&sm.empty[slot], ((g / kWsRing) & 1u) ^ 1u, &sm.abort)) return false;
    if (actA) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        const T* row = sm.tile + (2 * f + tb) * bufElems + rowSelf;
        const T2 xm = *reinterpret_cast<const T2*>(row - 2);
        const T2 xp = *reinterpret_cast<const T2*>(row + 2);
        const T2 ym1 = *reinterpret_cast<const T2*>(row - W);
        const T2 ym2 = *reinterpret_cast<const T2*>(row - 2 * W);
        const T2 yp1 = *reinterpret_cast<const T2*>(row + W);
        const T2 yp2 = *reinterpret_cast<const T2*>(row + 2 * W);
        T2 r;
        r.x = A::lap(c0[f].x, xm.y, c0[f].y, ym1.x, yp1.x, m1[f].x, p1[f].x, xm.x, xp.x,
                     ym2.x, yp2.x, m2[f].x, p2[f].x);
        r.y = A::lap(c0[f].y, c0[f].x, xp.x, ym1.y, yp1.y, m1[f].y, p1[f].y, xm.y, xp.y,
                     ym2.y, yp2.y, m2[f].y, p2[f].y);
        sm.ring[slot][f][tid] = r;
      }
    }
    mbar_arrive(&sm.full[slot]);
    ++g;
    return true;
  };
  // unrolled by the queue length so the five z-values never move
  bool ok = true;
  for (int kk = 0;;) {
    if (!(ok = plane(kk, qa, qb, qc, qd, qe))) break;
    if (++kk >= it.nzr) break;
    if (!(ok = plane(kk, qb, qc, qd, qe, qa))) break;
    if (++kk >= it.nzr) break;
    if (!(ok = plane(kk, qc, qd, qe, qa, qb))) break;
    if (++kk >= it.nzr) break;
    if (!(ok = plane(kk, qd, qe, qa, qb, qc))) break;
    if (++kk >= it.nzr) break;
    if (!(ok = plane(kk, qe, qa, qb, qc, qd))) break;
    if (++kk >= it.nzr) break;
  }
  cp_async_wait_all();
  return ok;
}

// Consumer role for one work item (threads 256..): pairs ctid + j *
// kWsConsumers (j < kWsPairs) of the tile.  For every plane it calls
//   epi.point(idx, pw, rA, rB, actB, x, y, k)
// as run_items does.  stall != 0 (failure-detection tests only):
// the consumers never release a slot, so the producers' wait for a free slot
// runs out.  Returns false if a wait gave up.
template <class Epi, class S>
__device__ __forceinline__ bool ws_consume(const DItem& it, const DBox& bx, S& sm,
                                           unsigned& err, unsigned& g, Epi& epi, int stall) {
  using A = typename S::Arith;
  static_assert(S::kNF == Epi::NF, "staging and epilogue disagree on the pointwise fields");
  using T = typename A::T;
  using T2 = typename A::T2;
  const int ctid = threadIdx.x - kWsProducers;
  const int txh = it.txh;
  const int pz = (int)bx.pz, py = (int)bx.py, off0 = (int)bx.off;
#ifdef SC_BOUNDS_CHECK
  const int blk0 = off0 - 2 - 2 * py - 2 * pz;
  const int blk1 = off0 - 3 + py + (bx.ny + 1) * py + (bx.nz + 1) * pz;
  auto ck = [&](int i) {
    if (i < blk0 || i + 1 > blk1) {
      err |= kErrBounds;
      return off0;
    }
    return i;
  };
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
  int t[kWsPairs], gxs[kWsPairs], gys[kWsPairs], op[kWsPairs], oi[kWsPairs];
  bool actA[kWsPairs], actB[kWsPairs];
#pragma unroll
  for (int j = 0; j < kWsPairs; ++j) {
    t[j] = ctid + kWsConsumers * j;
    const int lx = t[j] % txh, ly = t[j] / txh;
    gxs[j] = it.x0 + 2 * lx;
    gys[j] = it.y0 + ly;
    actA[j] = gxs[j] < bx.nx && gys[j] < bx.ny;
    actB[j] = gxs[j] + 1 < bx.nx && gys[j] < bx.ny;
    op[j] = off0 + (actA[j] ? gxs[j] + gys[j] * py : 0) + it.z0 * pz;
    oi[j] = op[j];
  }
  // the pointwise fields of pair j on the next plane, by cp.async
  auto stage_one = [&](int buf, int j) {
    if (actA[j]) {
#pragma unroll
      for (int f = 0; f < Epi::NF; ++f) cp_async16(&sm.pw[buf][f][t[j]], epi.f[f] + ck(op[j]));
    }
    op[j] += pz;
  };
  auto hand = [&](int j, int k, const double2 (&pw)[Epi::NF], unsigned slot) {
    T rA[2], rB[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const T2 s = sm.ring[slot][f][t[j]];
      rA[f] = s.x;
      rB[f] = s.y;
    }
    epi.point(oi[j], pw, rA, rB, actB[j], gxs[j], gys[j], k);
  };
  bool ok = true;
  if (S::kNB == 2) {
    // both pairs one plane ahead in one commit group per plane
    auto stage_pw = [&](int buf) {
#pragma unroll
      for (int j = 0; j < kWsPairs; ++j) stage_one(buf, j);
      cp_async_commit();
    };
    stage_pw(g & 1);
    for (int kk = 0; kk < it.nzr; ++kk) {
      const int k = it.z0 + kk;
      const int pb = (int)(g & 1u);
      if (kk + 1 < it.nzr)
        stage_pw(pb ^ 1);
      else
        cp_async_commit();
      cp_async_wait_one();  // this thread's pointwise values of plane k have landed
      const unsigned slot = g % kWsRing;
      if (!(ok = mbar_wait(&sm.full[slot], (g / kWsRing) & 1u, &sm.abort))) break;
#pragma unroll
      for (int j = 0; j < kWsPairs; ++j) {
        if (actA[j] && ok_pt(oi[j], gxs[j], gys[j], k, actB[j])) {
          double2 pw[Epi::NF];
#pragma unroll
          for (int f = 0; f < Epi::NF; ++f) pw[f] = sm.pw[pb & (S::kNB - 1)][f][t[j]];
          hand(j, k, pw, slot);
        }
        oi[j] += pz;
      }
      if (!stall) mbar_arrive(&sm.empty[slot]);
      ++g;
    }
  } else {
    // one buffer: one commit group per pair and plane; a pair's values are
    // copied to registers, its next plane is requested, then its epilogue
    // runs (the oldest pending group is always the next pair's)
#pragma unroll
    for (int j = 0; j < kWsPairs; ++j) {
      stage_one(0, j);
      cp_async_commit();
    }
    for (int kk = 0; kk < it.nzr; ++kk) {
      const int k = it.z0 + kk;
      const unsigned slot = g % kWsRing;
      if (!(ok = mbar_wait(&sm.full[slot], (g / kWsRing) & 1u, &sm.abort))) break;
#pragma unroll
      for (int j = 0; j < kWsPairs; ++j) {
        cp_async_wait_n<kWsPairs - 1>();  // pair j's values of plane k have landed
        double2 pw[Epi::NF];
#pragma unroll
        for (int f = 0; f < Epi::NF; ++f) pw[f] = sm.pw[0][f][t[j]];
        if (kk + 1 < it.nzr) stage_one(0, j);
        cp_async_commit();
        if (actA[j] && ok_pt(oi[j], gxs[j], gys[j], k, actB[j])) hand(j, k, pw, slot);
        oi[j] += pz;
      }
      if (!stall) mbar_arrive(&sm.empty[slot]);
      ++g;
    }
  }
  cp_async_wait_all();
  return ok;
}

}  // namespace dev
}  // namespace sc
