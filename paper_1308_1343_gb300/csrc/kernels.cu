// Kernels and their launchers.  See kernels.cuh for the traversal and the
// two arithmetic forms of the Laplacian sum.
//
// RK4 in nested form.  For the linear autonomous system y' = A y,
// A(u, pi) = (pi, c2 * L u), one classic RK4 step equals
//     y_new = (I + dt A + (dt A)^2/2 + (dt A)^3/6 + (dt A)^4/24) y,
// which the stage kernels evaluate as
//     w_0 = y,  w_s = y + g_s A w_{s-1},  g = (dt/4, dt/3, dt/2, dt),
//     y_new = w_4,
// i.e.  w_s.u  = y.u  + g_s * w_{s-1}.pi
//       w_s.pi = y.pi + g_s * c2 * (L w_{s-1}.u).
// Each stage is one fused pass: the stencil of w_{s-1}.u, two FMAs per
// point, and no K accumulators (26 instead of 38 doubles moved per point per
// step).  The pass kernels (pair_kernel) take two stages per pass, forming
// L w_1.u and L w_3.u by linearity from the stencils of the pass's two
// fields (15 doubles per point per step; see PairEpi).
#include "kernels.cuh"
#include "kernels_ws.cuh"
#include "launch.hpp"

namespace sc {
namespace dev {

constexpr int NT = 256;

// ---------------------------------------------------------------------------
// Ghost gather: dst[ghost point] = src[owner point], every rectangle copy of
// the exchange list, one launch.
// ---------------------------------------------------------------------------

template <bool TWO>
__global__ void __launch_bounds__(kGatherChunk) gather_kernel(
    const DRect* __restrict__ rects, const DChunk* __restrict__ chunks, int nchunks, double* f,
    double* g, unsigned* clear, int nclear) {
  // exponent slots that the next kernel accumulates into start at zero
  if (clear && blockIdx.x == 0)
    for (int d = threadIdx.x; d < nclear; d += blockDim.x) clear[d] = 0u;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const int p = ch.first + (int)threadIdx.x;
    const int ux = r.pairs ? r.ex >> 1 : r.ex;  // units per row: pairs or points
    if (p < ux * r.ey * r.ez) {
      const int t = p / ux;
      const int x = (p - t * ux) << r.pairs;
      const int z = t / r.ey;
      const int y = t - z * r.ey;
      // offsets fit 32 bits: a field holds fewer than 2^31 doubles
      const int dst = (int)r.dst + x + y * (int)r.dpy + z * (int)r.dpz;
      const int src = (int)r.src + x + y * (int)r.spy + z * (int)r.spz;
      if (r.pairs) {
        st2(f + dst, ld2(f + src));
        if (TWO) st2(g + dst, ld2(g + src));
      } else {
        f[dst] = f[src];
        if (TWO) g[dst] = g[src];
      }
    }
  }
}

// Exchange of a distributed level across ranks: PACK copies the points of
// every DXfer rectangle of two fields into the contiguous buffer (the second
// field `second` doubles after the first); otherwise the buffer is written
// back into the rectangles (ghost points of local boxes) and, if emax is not
// NULL, the largest biased exponent of what was written raises the exponent
// bounds emax[dom] (first field) and emax[ndom + dom] (second field) that
// the next pass reads.  One chunk of one rectangle per CTA iteration.
template <bool PACK>
__global__ void __launch_bounds__(kGatherChunk) xfer_kernel(
    const DXfer* __restrict__ xs, const DChunk* __restrict__ chunks, int nchunks, double* f,
    double* g, double* buf, unsigned* emax, int ndom) {
  __shared__ unsigned red[2 * kGatherChunk / 32];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DXfer r = xs[ch.rect];
    const int p = ch.first + (int)threadIdx.x;
    unsigned ea = 0u, eb = 0u;
    if (p < r.ex * r.ey * r.ez) {
      const int t = p / r.ex;
      const int x = p - t * r.ex;
      const int z = t / r.ey;
      const int y = t - z * r.ey;
      const long long fi = r.fld + x + y * r.fpy + z * r.fpz;
      const long long bi = r.buf + p;
      if (PACK) {
        buf[bi] = f[fi];
        buf[bi + r.second] = g[fi];
      } else {
        const double a = buf[bi], b = buf[bi + r.second];
        f[fi] = a;
        g[fi] = b;
        ea = biased_exp(a);
        eb = biased_exp(b);
      }
    }
    if (!PACK && emax) cta_max2_to(ea, eb, emax + r.dom, emax + ndom + r.dom, red);
  }
}

// Largest biased exponent of the field over the rectangles, per domain.
__global__ void __launch_bounds__(256) maxexp_kernel(const DRect* __restrict__ rects,
                                                     const DChunk* __restrict__ chunks,
                                                     int nchunks, const double* __restrict__ f,
                                                     unsigned* emax, unsigned* err) {
  __shared__ unsigned red[32];
  unsigned bad = 0;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const int n = r.ex * r.ey * r.ez;
    const int end = min(ch.first + kChunk, n);
    unsigned m = 0;
    for (int p = ch.first + threadIdx.x; p < end; p += blockDim.x) {
      const int x = p % r.ex;
      const int t = p / r.ex;
      const int y = t % r.ey;
      const int z = t / r.ey;
      m = max(m, biased_exp(f[r.src + x + y * r.spy + z * r.spz]));
    }
    if (m >= 0x7ffu) bad |= kErrNonFinite;
    cta_max_to(m, emax + r.dom, red);
  }
  if (bad) atomicOr(err, bad);
}

// out = a * b on the rectangles (interior points); optional exponent max.
template <bool TRACK>
__global__ void __launch_bounds__(256) mul_kernel(const DRect* __restrict__ rects,
                                                  const DChunk* __restrict__ chunks, int nchunks,
                                                  const double* __restrict__ a,
                                                  const double* __restrict__ b, double* out,
                                                  unsigned* emax) {
  __shared__ unsigned red[32];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const int n = r.ex * r.ey * r.ez;
    const int end = min(ch.first + kChunk, n);
    unsigned m = 0;
    for (int p = ch.first + threadIdx.x; p < end; p += blockDim.x) {
      const int x = p % r.ex;
      const int t = p / r.ex;
      const int y = t % r.ey;
      const int z = t / r.ey;
      const long long i = r.src + x + y * r.spy + z * r.spz;
      const double v = (a ? a[i] : 1.0) * b[i];
      out[i] = v;
      if (TRACK) m = max(m, biased_exp(v));
    }
    if (TRACK) cta_max_to(m, emax + r.dom, red);
  }
}

// q_a = c2 * fac[2 dom], q_b = c2 * fac[2 dom + 1] on interior points: the
// wave speed pre-scaled by dt / (12 h^2) and (dt/3) / (12 h^2) for the
// stage kernels of one run of steps.
__global__ void __launch_bounds__(256) qprep_kernel(const DRect* __restrict__ rects,
                                                    const DChunk* __restrict__ chunks,
                                                    int nchunks, const double* __restrict__ c2,
                                                    double* qa, double* qb,
                                                    const double* __restrict__ fac) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const double fa = fac[2 * r.dom], fb = fac[2 * r.dom + 1];
    const int n = r.ex * r.ey * r.ez;
    const int end = min(ch.first + kChunk, n);
    for (int p = ch.first + threadIdx.x; p < end; p += blockDim.x) {
      const int x = p % r.ex;
      const int t = p / r.ex;
      const int y = t % r.ey;
      const int z = t / r.ey;
      const long long i = r.src + x + y * r.spy + z * r.spz;
      const double v = c2[i];
      qa[i] = v * fa;
      qb[i] = v * fb;
    }
  }
}

// Misfit: per chunk, 1/2 sum (u - uo)^2 h^3 into partial[c] (fixed-order
// tree), and seed = h^3 (u - uo).
__global__ void __launch_bounds__(256) misfit_kernel(const DRect* __restrict__ rects,
                                                     const DChunk* __restrict__ chunks,
                                                     int nchunks, const double* __restrict__ u,
                                                     const double* __restrict__ uo,
                                                     double* seed, const double* __restrict__ h3,
                                                     double* partial) {
  __shared__ double red[256];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const double w = h3[r.dom];
    const int n = r.ex * r.ey * r.ez;
    const int end = min(ch.first + kChunk, n);
    double s = 0.0;
    for (int p = ch.first + threadIdx.x; p < end; p += blockDim.x) {
      const int x = p % r.ex;
      const int t = p / r.ex;
      const int y = t % r.ey;
      const int z = t / r.ey;
      const long long i = r.src + x + y * r.spy + z * r.spz;
      const double d = u[i] - uo[i];
      s += 0.5 * w * (d * d);
      if (seed) seed[i] = w * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
      if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[c] = red[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) sum_kernel(const double* __restrict__ partial, int n,
                                                  double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------------------
// Per-item setup shared by the stencil kernels
// ---------------------------------------------------------------------------

template <class A>
__device__ __forceinline__ A make_arith(const unsigned* emax_in, int dom, unsigned& err) {
  A a;
  if (A::kFixed) {
    const unsigned E = emax_in[dom];
    if (E >= 0x7ffu) err |= kErrNonFinite;
    // E >= 64 keeps every rescaled sum a normal number (fields below
    // 2^-958 are then represented to 2^-1013 absolute)
    a.E = (int)min(max(E, 64u), 0x7feu);
  }
  return a;
}


__device__ __forceinline__ void clear_slot(unsigned* slot, int ndom) {
  if (slot && blockIdx.x == 0)
    for (int d = threadIdx.x; d < ndom; d += blockDim.x) slot[d] = 0u;
}

// ---------------------------------------------------------------------------
// Forward stage: w_out = (y.u + g w_in.pi, y.pi + g c2 L w_in.u)
// ---------------------------------------------------------------------------

template <class A, bool RECORD>
struct FwdEpi {
  static constexpr int NF = 4;  // w_in.pi, y.u, y.pi, q (= c2 dt / (12 h^2), pre-scaled)
  const double* f[NF];
  double* wu_out;
  double* wp_out;
  double* __restrict__ lapw;
  A arith;
  int qk;          // stage factor 2^qk applied to q (1/4, 1/2, 1; 1/3 lives in q)
  double g, lw;    // g_s; scale of the recorded C_s L w (adjoint constant included)
  unsigned emax;

  __device__ __forceinline__ void point(int i, const double2* pw, typename A::T rA,
                                        typename A::T rB, bool actB, int, int, int) {
    const double2 wp = pw[0], u0 = pw[1], p0 = pw[2], q = pw[3];
    const double dA = arith.scaled(rA, qk), dB = arith.scaled(rB, qk);
    double2 un, pn;
    un.x = fma(g, wp.x, u0.x);
    un.y = fma(g, wp.y, u0.y);
    pn.x = fma(q.x, dA, p0.x);
    pn.y = fma(q.y, dB, p0.y);
    if (actB) {
      st2(wu_out + i, un);
      st2(wp_out + i, pn);
      if (RECORD) st2(lapw + i, make_double2(dA * lw, dB * lw));
    } else {
      wu_out[i] = un.x;
      wp_out[i] = pn.x;
      if (RECORD) lapw[i] = dA * lw;
    }
    if (A::kFixed) {
      emax = max(emax, biased_exp(un.x));
      if (actB) emax = max(emax, biased_exp(un.y));
    }
  }
};

// ASYNC: raw column and halo values staged by cp.async (62 KB of shared
// memory, 3 CTAs per SM) instead of in registers (46 KB, 4 CTAs per SM); the
// tuner picks one per level (sc_level_set_staging)
template <class A, bool RECORD, bool ASYNC>
__global__ void __launch_bounds__(NT, ASYNC ? 3 : 4) fwd_stage_kernel(FwdArgs a) {
  __shared__ Smem<NT, A, 4, 1, false, ASYNC> smem;
  __shared__ unsigned red[NT / 32];
  if (A::kFixed) clear_slot(a.emax_clear, a.ndom);
  unsigned err = 0;
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const StageCoef cf = a.coef[bx.dom];
    const A arith = make_arith<A>(a.emax_in, bx.dom, err);
    FwdEpi<A, RECORD> epi{{a.wp_in, a.yu, a.yp, a.q}, a.wu_out, a.wp_out, a.lapw, arith,
                          a.qk, cf.gamma, cf.rec};
    epi.emax = 0;
    run_item<NT, A, FwdEpi<A, RECORD>, ASYNC>(it, bx, a.wu_in, arith, smem, err, epi);
    // ghost copies of the new w.u, the next stage's stencil input
    push_item<NT>(PushTab{a.push, a.push_gofs}, it, bx, a.wu_out);
    if (A::kFixed) cta_max_to(epi.emax, a.emax_out + bx.dom, red);
  }
  if (err) atomicOr(a.err, err);
}

// ---------------------------------------------------------------------------
// Two RK4 stages per pass
// ---------------------------------------------------------------------------
//
// Only the u-component passes through the stencil, and w_s.u is pointwise in
// (y.u, w_{s-1}.pi).  So by linearity of L
//     L w_1.u = L y.u + g_1 L y.pi,     L w_3.u = L y.u + g_3 L w_2.pi,
// and a step splits into two passes whose stencils all have radius 2:
//   pass A (stages 1, 2), stencils of y.u and y.pi:
//     w_1.pi = y.pi + g_1 c2 L y.u        w_2.u  = y.u + g_2 w_1.pi
//     w_2.pi = y.pi + g_2 c2 (L y.u + g_1 L y.pi),   and it stores L y.u;
//   pass B (stages 3, 4), stencils of w_2.u and w_2.pi:
//     w_3.pi = y.pi + g_3 c2 L w_2.u      y.u   <- y.u + g_4 w_3.pi
//     y.pi  <- y.pi + g_4 c2 (L y.u + g_3 L w_2.pi)   (in place).
// Per point and step: 2 FP64 FMAs and one int->FP64 conversion per stage as
// in the one-stage kernels, but 15 instead of 26 doubles moved (A: read y.u,
// y.pi, q, q/3; write w_2, L y.u.  B: read w_2, y, q, L y.u; write y).
// Results differ from the one-stage form by rounding only.

template <class A, bool SECOND, bool RECORD>
struct PairEpi {
  static constexpr int NF = 4;  // y.u, y.pi, q = c2 dt/(12 h^2), then A: q/3, B: L y.u
  static constexpr bool kDefer = SECOND;  // measured: faster for pass B only
  const double* f[NF];
  double* out_u;
  double* out_p;
  double* __restrict__ ly;  // pass A: 12 h^2 L y.u
  double* __restrict__ r0;  // RECORD: C_s L w_{s-1}.u of the pass's two stages
  double* __restrict__ r1;
  A a0, a1;                 // arithmetic of the two stencil fields
  double ga, gb;            // A: g_1, g_2.  B: g_3, g_4
  double c0, c1;            // recording scales of the two stages
  unsigned eu, ep;

  // one point: s0, s1 the two stencil sums, x the pointwise fields; q0, q1
  // the recorded values (the stage kernel's C_s L w_{s-1}.u, same scaling)
  __device__ __forceinline__ void one(typename A::T s0, typename A::T s1, double u0, double p0,
                                      double q, double x, double& un, double& pn, double& lyv,
                                      double& q0, double& q1) const {
    if (!SECOND) {
      double dU, dU4;                      // 12 h^2 L y.u, and / 4
      a0.scaled2(s0, 0, -2, dU, dU4);
      const double dP = a1.scaled(s1, 0);  // 12 h^2 L y.pi
      const double w1p = fma(q, dU4, p0);
      const double lw1 = fma(ga, dP, dU);  // 12 h^2 L w_1.u
      un = fma(gb, w1p, u0);
      pn = fma(x, lw1, p0);
      lyv = dU;
      if (RECORD) {
        q0 = dU4 * c0;
        q1 = lw1 * c1;
      }
    } else {
      const double dA = a0.scaled(s0, -1);  // 12 h^2 L w_2.u * 1/2
      const double w3p = fma(q, dA, p0);
      const double lw3 = fma(ga, a1.scaled(s1, 0), x);  // 12 h^2 L w_3.u
      un = fma(gb, w3p, u0);
      pn = fma(q, lw3, p0);
      if (RECORD) {
        q0 = dA * c0;
        q1 = lw3 * c1;
      }
    }
  }

  __device__ __forceinline__ void point(int i, const double2* pw,
                                        const typename A::T (&rA)[2],
                                        const typename A::T (&rB)[2], bool actB, int, int,
                                        int) {
    const double2 u0 = pw[0], p0 = pw[1], q = pw[2], x = pw[3];
    double2 un, pn, lv, q0, q1;
    one(rA[0], rA[1], u0.x, p0.x, q.x, x.x, un.x, pn.x, lv.x, q0.x, q1.x);
    one(rB[0], rB[1], u0.y, p0.y, q.y, x.y, un.y, pn.y, lv.y, q0.y, q1.y);
    if (actB) {
      // pass A's outputs go out with an evict-first hint (measured: 4 %
      // faster; pass B was 3 % slower with it)
      if (!SECOND) {
        st2cs(out_u + i, un);
        st2cs(out_p + i, pn);
        st2cs(ly + i, lv);
      } else {
        st2(out_u + i, un);
        st2(out_p + i, pn);
      }
      if (RECORD) {
        st2(r0 + i, q0);
        st2(r1 + i, q1);
      }
    } else {
      out_u[i] = un.x;
      out_p[i] = pn.x;
      if (!SECOND) ly[i] = lv.x;
      if (RECORD) {
        r0[i] = q0.x;
        r1[i] = q1.x;
      }
    }
    if (A::kFixed) {
      eu = max(eu, biased_exp(un.x));
      ep = max(ep, biased_exp(pn.x));
      if (actB) {
        eu = max(eu, biased_exp(un.y));
        ep = max(ep, biased_exp(pn.y));
      }
    }
  }
};

template <class A, bool SECOND, bool RECORD>
__global__ void __launch_bounds__(NT, 2) pair_kernel(PairArgs a) {
  __shared__ Smem<NT, A, 4, 2, SECOND> smem;
  __shared__ unsigned red[2 * NT / 32];
  unsigned err = 0;
  const double* const F[2] = {a.s0, a.s1};
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const A ar[2] = {make_arith<A>(a.emax_in, bx.dom, err),
                     make_arith<A>(a.emax_in + a.ndom, bx.dom, err)};
    const int s0 = SECOND ? 2 : 0;  // stage coefficients g_{s0+1}, g_{s0+2}
    const StageCoef* ca = a.coef + s0 * a.ndom + bx.dom;
    const StageCoef* cb = ca + a.ndom;
    PairEpi<A, SECOND, RECORD> epi{{a.yu, a.yp, a.q, a.x}, a.out_u, a.out_p, a.ly, a.rec0,
                                   a.rec1, ar[0], ar[1], ca->gamma, cb->gamma,
                                   RECORD ? ca->rec : 0.0, RECORD ? cb->rec : 0.0, 0u, 0u};
    run_items<NT, 2>(it, bx, F, ar, smem, err, epi);
    if (A::kFixed)
      cta_max2_to(epi.eu, epi.ep, a.emax_out + bx.dom, a.emax_out + a.ndom + bx.dom, red);
  }
  if (err) atomicOr(a.err, err);
}

// The same passes with the warp-specialised traversal (kernels_ws.cuh):
// producer warps form the sums, consumer warps run PairEpi on them.  Results
// are bit-identical to pair_kernel.
template <class A, bool SECOND, bool RECORD>
__global__ void __launch_bounds__(kWsThreads, 2) pair_ws_kernel(PairArgs a) {
  __shared__ WsSmem<A> sm;
  ws_init(sm);
  unsigned err = 0, g = 0;
  bool ok = true;
  // registers: producers take 96 and consumers give back to what is left of
  // the CTA's (48 of 80 per thread with 4 consumer warps)
  if (threadIdx.x < kWsProducers) {
    ws_producer_regs<96>();
    const double* const F[2] = {a.s0, a.s1};
    const XgTab xt{a.xg, a.xg_ofs, a.boxes};
    for (int i = blockIdx.x; i < a.nitems && ok; i += gridDim.x) {
      const DItem it = a.items[i];
      const DBox bx = a.boxes[it.box];
      const A ar[2] = {make_arith<A>(a.emax_in, bx.dom, err),
                       make_arith<A>(a.emax_in + a.ndom, bx.dom, err)};
      ok = ws_produce(it, bx, F, ar, sm, err, g, xt);
    }
  } else {
    ws_consumer_regs<96>();
    for (int i = blockIdx.x; i < a.nitems && ok; i += gridDim.x) {
      const DItem it = a.items[i];
      const DBox bx = a.boxes[it.box];
      unsigned e2 = 0;  // a bad bound is reported by the producers
      const A ar[2] = {make_arith<A>(a.emax_in, bx.dom, e2),
                       make_arith<A>(a.emax_in + a.ndom, bx.dom, e2)};
      const int s0 = SECOND ? 2 : 0;
      const StageCoef* ca = a.coef + s0 * a.ndom + bx.dom;
      const StageCoef* cb = ca + a.ndom;
      PairEpi<A, SECOND, RECORD> epi{{a.yu, a.yp, a.q, a.x}, a.out_u, a.out_p, a.ly, a.rec0,
                                     a.rec1, ar[0], ar[1], ca->gamma, cb->gamma,
                                     RECORD ? ca->rec : 0.0, RECORD ? cb->rec : 0.0, 0u, 0u};
      ok = ws_consume(it, bx, sm, err, g, epi, a.stall);
      // one verdict per warp before the warp-wide reduction (a lane whose
      // wait gave up must not leave the others in a collective)
      ok = __all_sync(0xffffffffu, ok);
      if (ok && A::kFixed) {
        // exponent bounds of the item's outputs: one atomicMax per warp
        const unsigned eu = __reduce_max_sync(0xffffffffu, epi.eu);
        const unsigned ep = __reduce_max_sync(0xffffffffu, epi.ep);
        if ((threadIdx.x & 31) == 0) {
          if (eu) atomicMax(a.emax_out + bx.dom, eu);
          if (ep) atomicMax(a.emax_out + a.ndom + bx.dom, ep);
        }
      }
    }
  }
  if (!ok) {
    reinterpret_cast<volatile int&>(sm.abort) = 1;
    err |= kErrTimeout;
  }
  if (err) atomicOr(a.err, err);
}

// ---------------------------------------------------------------------------
// out = L u
// ---------------------------------------------------------------------------

template <class A>
struct LapEpi {
  static constexpr int NF = 0;
  const double* f[1];
  double* out;
  A arith;
  double lw;
  __device__ __forceinline__ void point(int i, const double2*, typename A::T rA,
                                        typename A::T rB, bool actB, int, int, int) {
    const double dA = arith.scaled(rA, 0) * lw, dB = arith.scaled(rB, 0) * lw;
    if (actB)
      st2(out + i, make_double2(dA, dB));
    else
      out[i] = dA;
  }
};

template <class A>
__global__ void __launch_bounds__(NT, 4) lap_kernel(LapArgs a) {
  __shared__ Smem<NT, A, 0> smem;
  unsigned err = 0;
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const A arith = make_arith<A>(a.emax_in, bx.dom, err);
    LapEpi<A> epi{{nullptr}, a.out, arith, a.inv12h2[bx.dom]};
    run_item<NT>(it, bx, a.u, arith, smem, err, epi);
  }
  if (err) atomicOr(a.err, err);
}

// ---------------------------------------------------------------------------
// Adjoint of one nested-RK4 step.  With M = L(c2 .), the reverse of
// w_s = y + g_s A w_{s-1} (A^T(a, b) = (L(c2 b), a), L symmetric) applied to
// the adjoint (a, b) of the step's output needs four applications of M:
//   P4 = M b,  P3 = M a,  P2 = M P4,  P1 = M P3,
// and then, with G4 = g4, G34 = g3 g4, G234 = g2 g3 g4, G1234 = g1 g2 g3 g4:
//   ybar.u  = a + G4 P4 + G34 P3 + G234 P2 + G1234 P1
//   ybar.pi = b + G4 a + G34 P4 + G234 P3 + G1234 P2
//   c2bar  += G4 b Lw3 + G34 a Lw2 + G234 P4 Lw1 + G1234 P3 Lw0
// (Lw_{s-1} = L w_{s-1}.u of forward stage s).  The kernels work with the
// unscaled sums Phat = 12 h^2 P; all constant factors (the G's, powers of
// 1/(12 h^2)) are folded into per-domain coefficients, and the forward pass
// records Q_s = C_s Lw_{s-1} already multiplied by its constant.
//   adj2 first  : Phat4, Phat3 = L^ z for z = c2 b, c2 a, and z' = c2 Phat
//   adj2 second : Phat2 = L^ (c2 Phat4), Phat1 = L^ (c2 Phat3)
//   adj_combine : the combination above, pointwise; it also writes the next
//                 (earlier) step's stencil inputs c2 ybar.pi and c2 ybar.u
// ---------------------------------------------------------------------------

// The four applications of M as two passes over two stencil fields each:
//   adj2 first  : (Phat4, Phat3) = L^ (c2 b, c2 a), and (c2 Phat4, c2 Phat3)
//                 with their ghosts pushed (the second pass's inputs);
//   adj2 second : (Phat2, Phat1) = L^ (c2 Phat4, c2 Phat3).
template <class A, bool SECOND>
struct Adj2Epi {
  static constexpr int NF = SECOND ? 0 : 1;  // c2
  static constexpr bool kHaloSplit = true;  // measured: faster here
  const double* f[1];
  double* __restrict__ p0;
  double* __restrict__ p1;
  double* __restrict__ z0;
  double* __restrict__ z1;
  A a0, a1;
  unsigned e0, e1;
  __device__ __forceinline__ void point(int i, const double2* pw,
                                        const typename A::T (&rA)[2],
                                        const typename A::T (&rB)[2], bool actB, int, int,
                                        int) {
    const double2 q0 = make_double2(a0.scaled(rA[0], 0), a0.scaled(rB[0], 0));
    const double2 q1 = make_double2(a1.scaled(rA[1], 0), a1.scaled(rB[1], 0));
    double2 y0, y1;
    if (!SECOND) {
      const double2 c = pw[0];
      y0 = make_double2(c.x * q0.x, c.y * q0.y);
      y1 = make_double2(c.x * q1.x, c.y * q1.y);
    }
    if (actB) {
      st2(p0 + i, q0);
      st2(p1 + i, q1);
      if (!SECOND) {
        st2(z0 + i, y0);
        st2(z1 + i, y1);
      }
    } else {
      p0[i] = q0.x;
      p1[i] = q1.x;
      if (!SECOND) {
        z0[i] = y0.x;
        z1[i] = y1.x;
      }
    }
    if (A::kFixed && !SECOND) {
      e0 = max(e0, biased_exp(y0.x));
      e1 = max(e1, biased_exp(y1.x));
      if (actB) {
        e0 = max(e0, biased_exp(y0.y));
        e1 = max(e1, biased_exp(y1.y));
      }
    }
  }
};

template <class A, bool SECOND>
__global__ void __launch_bounds__(NT, 2) adj2_kernel(Adj2Args a) {
  __shared__ Smem<NT, A, SECOND ? 0 : 1, 2> smem;
  __shared__ unsigned red[2 * NT / 32];
  if (A::kFixed) clear_slot(a.emax_clear, 2 * a.ndom);
  unsigned err = 0;
  const double* const F[2] = {a.z0_in, a.z1_in};
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const A ar[2] = {make_arith<A>(a.emax_in, bx.dom, err),
                     make_arith<A>(a.emax_in + a.ndom, bx.dom, err)};
    Adj2Epi<A, SECOND> epi{{a.c2}, a.p0_out, a.p1_out, a.z0_out, a.z1_out, ar[0], ar[1],
                           0u, 0u};
    run_items<NT, 2>(it, bx, F, ar, smem, err, epi);
    if (!SECOND) {
      const PushTab pt{a.push, a.push_gofs};
      push_item<NT>(pt, it, bx, a.z0_out);  // the second pass's stencil inputs
      push_item<NT>(pt, it, bx, a.z1_out);
      if (A::kFixed)
        cta_max2_to(epi.e0, epi.e1, a.emax_out + bx.dom, a.emax_out + a.ndom + bx.dom, red);
    }
  }
  if (err) atomicOr(a.err, err);
}

// The adjoint step in two warp-specialised passes, without the pointwise
// combination kernel: each output below is formed by the same FMAs in the
// same nesting as adj_combine_kernel forms it (the first pass rounds the inner
// part, the second adds the outer terms), and Phat4..Phat1, c2 Phat4, c2 Phat3
// are those of adj2_kernel, so the gradients are bit-identical to the
// one-role path.  The combination's FP64 work runs in the consumer warps,
// beside the producers' integer work.
template <class A, bool SECOND>
struct AdjWsEpi {
  // first: c2, a, b, c2bar, Q1..Q4 (one buffer, each pair's next plane as
  // soon as its values are read); second: ybar.u part, ybar.pi part, c2
  static constexpr int NF = SECOND ? 3 : 8;
  const double* f[NF];
  double* yu;
  double* yp;
  double* cb;
  double* zo0;
  double* zo1;
  A a0, a1;
  AdjCoef k;
  unsigned e0, e1;
  __device__ __forceinline__ void one(typename A::T s0, typename A::T s1, const double* v,
                                      double& z0, double& z1, double& ou, double& op,
                                      double& oc) const {
    const double Pa = a0.scaled(s0, 0), Pb = a1.scaled(s1, 0);
    if (!SECOND) {
      // Pa = Phat4, Pb = Phat3; v = c2, a, b, c2bar, Q1, Q2, Q3, Q4
      const double cc = v[0], av = v[1], bv = v[2];
      z0 = cc * Pa;
      z1 = cc * Pb;
      ou = fma(k.cu[1], Pb, fma(k.cu[0], Pa, av));
      op = fma(k.cp[2], Pb, fma(k.cp[1], Pa, fma(k.cp[0], av, bv)));
      oc = fma(Pb, v[4], fma(Pa, v[5], fma(av, v[6], fma(bv, v[7], v[3]))));
    } else {
      // Pa = Phat2, Pb = Phat1; v = ybar.u part, ybar.pi part, c2
      ou = fma(k.cu[3], Pb, fma(k.cu[2], Pa, v[0]));
      op = fma(k.cp[3], Pa, v[1]);
      z0 = v[2] * op;
      z1 = v[2] * ou;
      oc = 0.0;
    }
  }
  __device__ __forceinline__ void point(int i, const double2* pw,
                                        const typename A::T (&rA)[2],
                                        const typename A::T (&rB)[2], bool actB, int, int,
                                        int) {
    double va[NF], vb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      va[f] = pw[f].x;
      vb[f] = pw[f].y;
    }
    double2 z0, z1, ou, op, oc;
    one(rA[0], rA[1], va, z0.x, z1.x, ou.x, op.x, oc.x);
    one(rB[0], rB[1], vb, z0.y, z1.y, ou.y, op.y, oc.y);
    if (actB) {
      st2(zo0 + i, z0);
      st2(zo1 + i, z1);
      st2(yu + i, ou);
      st2(yp + i, op);
      if (!SECOND) st2(cb + i, oc);
    } else {
      zo0[i] = z0.x;
      zo1[i] = z1.x;
      yu[i] = ou.x;
      yp[i] = op.x;
      if (!SECOND) cb[i] = oc.x;
    }
    if (A::kFixed) {
      e0 = max(e0, biased_exp(z0.x));
      e1 = max(e1, biased_exp(z1.x));
      if (actB) {
        e0 = max(e0, biased_exp(z0.y));
        e1 = max(e1, biased_exp(z1.y));
      }
    }
  }
};

template <class A, bool SECOND>
__global__ void __launch_bounds__(kWsThreads, 2) adj_ws_kernel(AdjWsArgs a) {
  __shared__ WsSmem<A, SECOND ? 3 : 8, SECOND ? 2 : 1> sm;
  if (A::kFixed) clear_slot(a.emax_clear, 2 * a.ndom);
  ws_init(sm);
  unsigned err = 0, g = 0;
  bool ok = true;
  // the first pass's consumers hold eight pointwise fields: producers 88 there
  // (consumers 64 with 4 consumer warps)
  constexpr int kP = SECOND ? 96 : 88;
  if (threadIdx.x < kWsProducers) {
    ws_producer_regs<kP>();
    const double* const F[2] = {a.z0_in, a.z1_in};
    const XgTab xt{a.xg, a.xg_ofs, a.boxes};
    for (int i = blockIdx.x; i < a.nitems && ok; i += gridDim.x) {
      const DItem it = a.items[i];
      const DBox bx = a.boxes[it.box];
      const A ar[2] = {make_arith<A>(a.emax_in, bx.dom, err),
                       make_arith<A>(a.emax_in + a.ndom, bx.dom, err)};
      ok = ws_produce(it, bx, F, ar, sm, err, g, xt);
    }
  } else {
    ws_consumer_regs<kP>();
    for (int i = blockIdx.x; i < a.nitems && ok; i += gridDim.x) {
      const DItem it = a.items[i];
      const DBox bx = a.boxes[it.box];
      unsigned e2 = 0;  // a bad bound is reported by the producers
      AdjWsEpi<A, SECOND> epi;
      if (SECOND) {
        epi.f[0] = a.yu;
        epi.f[1] = a.yp;
        epi.f[2] = a.c2;
      } else {
        const double* fs[8] = {a.c2, a.yu, a.yp, a.c2bar, a.q1, a.q2, a.q3, a.q4};
#pragma unroll
        for (int f = 0; f < AdjWsEpi<A, SECOND>::NF; ++f) epi.f[f] = fs[f];
      }
      epi.yu = a.yu;
      epi.yp = a.yp;
      epi.cb = a.c2bar;
      epi.zo0 = a.z0_out;
      epi.zo1 = a.z1_out;
      epi.a0 = make_arith<A>(a.emax_in, bx.dom, e2);
      epi.a1 = make_arith<A>(a.emax_in + a.ndom, bx.dom, e2);
      epi.k = a.coef[bx.dom];
      epi.e0 = epi.e1 = 0u;
      ok = ws_consume(it, bx, sm, err, g, epi, a.stall);
      ok = __all_sync(0xffffffffu, ok);
      if (ok && A::kFixed) {
        const unsigned e0 = __reduce_max_sync(0xffffffffu, epi.e0);
        const unsigned e1 = __reduce_max_sync(0xffffffffu, epi.e1);
        if ((threadIdx.x & 31) == 0) {
          if (e0) atomicMax(a.emax_out + bx.dom, e0);
          if (e1) atomicMax(a.emax_out + a.ndom + bx.dom, e1);
        }
      }
    }
  }
  if (!ok) {
    reinterpret_cast<volatile int&>(sm.abort) = 1;
    err |= kErrTimeout;
  }
  if (err) atomicOr(a.err, err);
}

// The combination of one adjoint step, pointwise over interior points: one
// point per thread (chunks of kGatherChunk points), all fields distinct.  It
// streams 12 fields in and 5 out, so memory parallelism sets its speed: 32
// registers give 8 CTAs per SM (measured: faster than 40 registers and 6
// CTAs, and than two points per thread with 16-byte accesses).
template <bool FIXED>
__global__ void __launch_bounds__(kGatherChunk, 8) adj_combine_kernel(
    const DRect* __restrict__ rects, const DChunk* __restrict__ chunks, int nchunks,
    AdjCombineArgs a) {
  __shared__ unsigned red[32];
  double* __restrict__ yu = a.yu;
  double* __restrict__ yp = a.yp;
  double* __restrict__ cb = a.c2bar;
  double* __restrict__ xo = a.x_out;
  double* __restrict__ yo = a.y_out;
  const double* __restrict__ p4 = a.p4;
  const double* __restrict__ p3 = a.p3;
  const double* __restrict__ p2 = a.p2;
  const double* __restrict__ p1 = a.p1;
  const double* __restrict__ q1 = a.q1;
  const double* __restrict__ q2 = a.q2;
  const double* __restrict__ q3 = a.q3;
  const double* __restrict__ q4 = a.q4;
  const double* __restrict__ c2 = a.c2;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const AdjCoef k = a.coef[r.dom];
    const int p = ch.first + (int)threadIdx.x;
    unsigned mx = 0, my = 0;
    if (p < r.ex * r.ey * r.ez) {
      const int t = p / r.ex;
      const int x = p - t * r.ex;
      const int z = t / r.ey;
      const int y = t - z * r.ey;
      const int i = (int)r.src + x + y * (int)r.spy + z * (int)r.spz;
      const double av = yu[i], bv = yp[i];
      const double P4 = p4[i], P3 = p3[i], P2 = p2[i], P1 = p1[i];
      const double Q1 = q1[i], Q2 = q2[i], Q3 = q3[i], Q4 = q4[i], cbv = cb[i], cc = c2[i];
      const double ou = fma(k.cu[3], P1, fma(k.cu[2], P2, fma(k.cu[1], P3, fma(k.cu[0], P4, av))));
      const double op = fma(k.cp[3], P2, fma(k.cp[2], P3, fma(k.cp[1], P4, fma(k.cp[0], av, bv))));
      const double oc = fma(P3, Q1, fma(P4, Q2, fma(av, Q3, fma(bv, Q4, cbv))));
      const double ox = cc * op, oy = cc * ou;
      yu[i] = ou;
      yp[i] = op;
      cb[i] = oc;
      xo[i] = ox;
      yo[i] = oy;
      const int gx = r.x0 + x, gy = r.y0 + y, gz = r.z0 + z;
      const DBox bx = a.boxes[r.box];
      if (a.push_gofs &&
          (gx < 2 || gx >= bx.nx - 2 || gy < 2 || gy >= bx.ny - 2 || gz < 2 || gz >= bx.nz - 2)) {
        const PushTab pt{a.push, a.push_gofs};
        push_point(pt, r.box, gx, gy, gz, bx.nx, bx.ny, bx.nz, ox, xo);
        push_point(pt, r.box, gx, gy, gz, bx.nx, bx.ny, bx.nz, oy, yo);
      }
      if (FIXED) {
        mx = biased_exp(ox);
        my = biased_exp(oy);
      }
    }
    if (FIXED) {
      cta_max_to(mx, a.emax_x + r.dom, red);
      cta_max_to(my, a.emax_y + r.dom, red);
    }
  }
}

// ---------------------------------------------------------------------------
// Two-level hierarchy: prolongation and restriction
// ---------------------------------------------------------------------------
//
// Prolongation: cubic Lagrange interpolation along each axis as a tensor
// product (weights (-1, 9, 9, -1)/16 at odd fine indices, injection at even
// ones), of data interpolated linearly in time, (1 - alpha) old + alpha new,
// per coarse point.  The tensor product is applied as successive
// one-dimensional interpolations, along z, then y, then x, each a chain of
// fused multiply-adds (measured: 29 % faster than separately rounded products
// and sums; GB300's FP64 pipe bounds this kernel); a tile's points share the
// z- and y-interpolated intermediates (shared memory).  The result is the
// interpolant up to rounding: exact where every product and partial sum is
// (dyadic data), else within a few ulps of the data's scale.
// Each list entry holds points of one parity per axis, so a CTA runs one
// stencil shape.  At alpha != 0 the time interpolation is done once per
// coarse point by blend_kernel into scratch coarse fields (the same
// rounding).

// One-dimensional interpolation along an axis of parity P (1: odd index):
// 0 + w_0 v_0 + w_1 v_1 + w_2 v_2 + w_3 v_3 with w = (-1, 9, 9, -1)/16, the
// first product exact (a power of two) and the rest fused multiply-adds in
// that order; at an even index 0 + v_0.  The values are v_k = f[i + k *
// stride].
__device__ __forceinline__ double plus_zero(double v) {  // 0.0 + v
  return (__double_as_longlong(v) << 1) == 0 ? 0.0 : v;
}
template <int P>
__device__ __forceinline__ double interp1(const double* __restrict__ f, long long i,
                                          long long stride) {
  if (!P) return plus_zero(f[i]);
  double acc = plus_zero(__dmul_rn(-0.0625, f[i]));
  acc = __fma_rn(0.5625, f[i + stride], acc);
  acc = __fma_rn(0.5625, f[i + 2 * stride], acc);
  return __fma_rn(-0.0625, f[i + 3 * stride], acc);
}

// The tile of one prolongation entry: z interpolation of every coarse (y, x)
// column the tile's stencils touch, then y, then x, staged in shared memory.
template <int PX, int PY, int PZ>
__device__ __forceinline__ void prol_tile(const DProl& r, int x0, int y0, int z0, int nx, int ny,
                                          int nz, const double* __restrict__ du,
                                          const double* __restrict__ dp, double* __restrict__ fu,
                                          double* __restrict__ fp, double (*t1)[2], double (*t2)[2],
                                          unsigned& mu, unsigned& mp) {
  constexpr int NX = PX ? 4 : 1, NY = PY ? 4 : 1;
  // coarse index of the first stencil point of the tile's first target
  const int cx0 = (PX ? ((r.fx0 - 1) >> 1) - 1 : r.fx0 >> 1) + x0;
  const int cy0 = (PY ? ((r.fy0 - 1) >> 1) - 1 : r.fy0 >> 1) + y0;
  const int cz0 = (PZ ? ((r.fz0 - 1) >> 1) - 1 : r.fz0 >> 1) + z0;
  const int wx = nx + NX - 1, wy = ny + NY - 1;
  // along z: t1[(z * wy + j) * wx + i] for column (cx0 + i, cy0 + j)
  const int n1 = nz * wy * wx;
  for (int k = threadIdx.x; k < n1; k += blockDim.x) {
    const int i = k % wx, jz = k / wx;
    const int j = jz % wy, z = jz / wy;
    const long long c =
        r.cbase + (long long)(cz0 + z) * r.cpz + (long long)(cy0 + j) * r.cpy + cx0 + i;
    t1[k][0] = interp1<PZ>(du, c, r.cpz);
    t1[k][1] = interp1<PZ>(dp, c, r.cpz);
  }
  __syncthreads();
  // along y: t2[(z * ny + y) * wx + i]
  const int n2 = nz * ny * wx;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    const int i = k % wx, yz = k / wx;
    const int y = yz % ny, z = yz / ny;
    const int b = (z * wy + y) * wx + i;
    double a0, a1;
    if (!PY) {
      a0 = plus_zero(t1[b][0]);
      a1 = plus_zero(t1[b][1]);
    } else {
      a0 = plus_zero(__dmul_rn(-0.0625, t1[b][0]));
      a1 = plus_zero(__dmul_rn(-0.0625, t1[b][1]));
      a0 = __fma_rn(0.5625, t1[b + wx][0], a0);
      a1 = __fma_rn(0.5625, t1[b + wx][1], a1);
      a0 = __fma_rn(0.5625, t1[b + 2 * wx][0], a0);
      a1 = __fma_rn(0.5625, t1[b + 2 * wx][1], a1);
      a0 = __fma_rn(-0.0625, t1[b + 3 * wx][0], a0);
      a1 = __fma_rn(-0.0625, t1[b + 3 * wx][1], a1);
    }
    t2[k][0] = a0;
    t2[k][1] = a1;
  }
  __syncthreads();
  // along x, and the fine points
  const int n3 = nz * ny * nx;
  for (int k = threadIdx.x; k < n3; k += blockDim.x) {
    const int x = k % nx, yz = k / nx;
    const int y = yz % ny, z = yz / ny;
    const int b = (z * ny + y) * wx + x;
    double su, sp;
    if (!PX) {
      su = plus_zero(t2[b][0]);
      sp = plus_zero(t2[b][1]);
    } else {
      su = plus_zero(__dmul_rn(-0.0625, t2[b][0]));
      sp = plus_zero(__dmul_rn(-0.0625, t2[b][1]));
      su = __fma_rn(0.5625, t2[b + 1][0], su);
      sp = __fma_rn(0.5625, t2[b + 1][1], sp);
      su = __fma_rn(0.5625, t2[b + 2][0], su);
      sp = __fma_rn(0.5625, t2[b + 2][1], sp);
      su = __fma_rn(-0.0625, t2[b + 3][0], su);
      sp = __fma_rn(-0.0625, t2[b + 3][1], sp);
    }
    const long long o = r.dst + 2ll * (x0 + x) + 2ll * (y0 + y) * r.dpy + 2ll * (z0 + z) * r.dpz;
    fu[o] = su;
    fp[o] = sp;
    mu = max(mu, biased_exp(su));
    mp = max(mp, biased_exp(sp));
  }
  __syncthreads();  // the next tile reuses the buffers
}

__global__ void __launch_bounds__(256) prolong_kernel(
    const DProl* __restrict__ rects, const DChunk* __restrict__ tiles, int ntiles,
    const double* __restrict__ du, const double* __restrict__ dp, double* __restrict__ fu,
    double* __restrict__ fp, unsigned* emax) {
  __shared__ double t1[kProlTZ * (kProlTY + 3) * (kProlTX + 3)][2];
  __shared__ double t2[kProlTZ * kProlTY * (kProlTX + 3)][2];
  __shared__ unsigned red[2 * 256 / 32];
  unsigned mu = 0, mp = 0;
  for (int c = blockIdx.x; c < ntiles; c += gridDim.x) {
    const DChunk ch = tiles[c];
    const DProl r = rects[ch.rect];
    const int ntx = (r.ex + kProlTX - 1) / kProlTX, nty = (r.ey + kProlTY - 1) / kProlTY;
    const int tx = ch.first % ntx, tyz = ch.first / ntx;
    const int ty = tyz % nty, tz = tyz / nty;
    const int x0 = tx * kProlTX, y0 = ty * kProlTY, z0 = tz * kProlTZ;
    const int nx = min(kProlTX, r.ex - x0), ny = min(kProlTY, r.ey - y0);
    const int nz = min(kProlTZ, r.ez - z0);
    // one parity class per list entry: a uniform branch
    switch ((r.fx0 & 1) | ((r.fy0 & 1) << 1) | ((r.fz0 & 1) << 2)) {
      case 0: prol_tile<0, 0, 0>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      case 1: prol_tile<1, 0, 0>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      case 2: prol_tile<0, 1, 0>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      case 3: prol_tile<1, 1, 0>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      case 4: prol_tile<0, 0, 1>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      case 5: prol_tile<1, 0, 1>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      case 6: prol_tile<0, 1, 1>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
      default: prol_tile<1, 1, 1>(r, x0, y0, z0, nx, ny, nz, du, dp, fu, fp, t1, t2, mu, mp); break;
    }
  }
  // the fine level's exponent bounds of u and pi take the written values in
  if (emax) cta_max2_to(mu, mp, emax, emax + 1, red);
}

// out = (1 - alpha) a + alpha b on the rectangles, rounded step by step.
__global__ void __launch_bounds__(256) blend_kernel(const DRect* __restrict__ rects,
                                                    const DChunk* __restrict__ chunks,
                                                    int nchunks, const double* __restrict__ a0,
                                                    const double* __restrict__ a1,
                                                    const double* __restrict__ b0,
                                                    const double* __restrict__ b1, double alpha,
                                                    double* __restrict__ ao,
                                                    double* __restrict__ bo) {
  const double beta = 1.0 - alpha;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const int n = r.ex * r.ey * r.ez;
    const int end = min(ch.first + kChunk, n);
    for (int p = ch.first + threadIdx.x; p < end; p += blockDim.x) {
      const int t = p / r.ex;
      const int x = p - t * r.ex;
      const int z = t / r.ey;
      const int y = t - z * r.ey;
      const long long i = r.src + x + (long long)y * r.spy + (long long)z * r.spz;
      ao[i] = __dadd_rn(__dmul_rn(beta, a0[i]), __dmul_rn(alpha, a1[i]));
      bo[i] = __dadd_rn(__dmul_rn(beta, b0[i]), __dmul_rn(alpha, b1[i]));
    }
  }
}

// Restriction by injection: coarse point c takes the fine value at 2c.
__global__ void __launch_bounds__(kGatherChunk) restrict_kernel(
    const DRestr* __restrict__ rects, const DChunk* __restrict__ chunks, int nchunks,
    const double* __restrict__ fu, const double* __restrict__ fp, double* __restrict__ cu,
    double* __restrict__ cp, unsigned* emax) {
  __shared__ unsigned red[2 * kGatherChunk / 32];
  unsigned mu = 0, mp = 0;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRestr r = rects[ch.rect];
    const int p = ch.first + (int)threadIdx.x;
    if (p >= r.ex * r.ey * r.ez) continue;
    const int t = p / r.ex;
    const int x = p - t * r.ex;
    const int z = t / r.ey;
    const int y = t - z * r.ey;
    const long long d = r.dst + x + (long long)y * r.dpy + (long long)z * r.dpz;
    const long long s = r.src + 2ll * x + 2ll * y * r.spy + 2ll * z * r.spz;
    const double vu = fu[s], vp = fp[s];
    cu[d] = vu;
    cp[d] = vp;
    mu = max(mu, biased_exp(vu));
    mp = max(mp, biased_exp(vp));
  }
  // the coarse level's exponent bounds of u and pi take the written values in
  if (emax) cta_max2_to(mu, mp, emax, emax + 1, red);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

cudaError_t launch_gather(const DRect* rects, const DChunk* chunks, int nchunks, double* f,
                          int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  (void)grid;
  gather_kernel<false><<<nchunks, kGatherChunk, 0, s>>>(rects, chunks, nchunks, f, nullptr,
                                                         nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_gather2(const DRect* rects, const DChunk* chunks, int nchunks, double* f,
                           double* g, unsigned* clear, int nclear, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  gather_kernel<true><<<nchunks, kGatherChunk, 0, s>>>(rects, chunks, nchunks, f, g, clear,
                                                        nclear);
  return cudaGetLastError();
}

cudaError_t launch_maxexp(const DRect* rects, const DChunk* chunks, int nchunks,
                          const double* f, unsigned* emax, unsigned* err, int grid,
                          cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  maxexp_kernel<<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, f, emax, err);
  return cudaGetLastError();
}

cudaError_t launch_mul(const DRect* rects, const DChunk* chunks, int nchunks, const double* a,
                       const double* b, double* out, unsigned* emax, int grid,
                       cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  if (emax)
    mul_kernel<true><<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, a, b, out, emax);
  else
    mul_kernel<false><<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, a, b, out,
                                                         nullptr);
  return cudaGetLastError();
}

cudaError_t launch_qprep(const DRect* rects, const DChunk* chunks, int nchunks,
                         const double* c2, double* qa, double* qb, const double* fac, int grid,
                         cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  qprep_kernel<<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, c2, qa, qb, fac);
  return cudaGetLastError();
}

cudaError_t launch_misfit(const DRect* rects, const DChunk* chunks, int nchunks,
                          const double* u, const double* uo, double* seed, const double* h3,
                          double* partial, double* loss, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  misfit_kernel<<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, u, uo, seed, h3,
                                                   partial);
  sum_kernel<<<1, 256, 0, s>>>(partial, nchunks, loss);
  return cudaGetLastError();
}

// Four 46 KB stage CTAs, or two 108 KB pass-B CTAs, per SM need the largest
// shared-memory carveout.
template <class K>
void prefer_shared(K kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

static void set_carveouts() {
  static bool done = false;
  if (done) return;
  done = true;
  prefer_shared(fwd_stage_kernel<Fixed, true, false>);
  prefer_shared(fwd_stage_kernel<Fixed, false, false>);
  prefer_shared(fwd_stage_kernel<Fp64, true, false>);
  prefer_shared(fwd_stage_kernel<Fp64, false, false>);
  prefer_shared(fwd_stage_kernel<Fixed, true, true>);
  prefer_shared(fwd_stage_kernel<Fixed, false, true>);
  prefer_shared(fwd_stage_kernel<Fp64, true, true>);
  prefer_shared(fwd_stage_kernel<Fp64, false, true>);
  prefer_shared(lap_kernel<Fixed>);
  prefer_shared(lap_kernel<Fp64>);
  // pass B keeps three planes of pointwise fields: two 108 KB CTAs per SM
  prefer_shared(pair_kernel<FixedI, false, false>);
  prefer_shared(pair_kernel<FixedI, true, false>);
  prefer_shared(pair_kernel<Fp64, false, false>);
  prefer_shared(pair_kernel<Fp64, true, false>);
  prefer_shared(pair_kernel<FixedI, false, true>);
  prefer_shared(pair_kernel<FixedI, true, true>);
  prefer_shared(pair_kernel<Fp64, false, true>);
  prefer_shared(pair_kernel<Fp64, true, true>);
  prefer_shared(pair_ws_kernel<FixedI, false, false>);
  prefer_shared(pair_ws_kernel<FixedI, true, false>);
  prefer_shared(pair_ws_kernel<Fp64, false, false>);
  prefer_shared(pair_ws_kernel<Fp64, true, false>);
  prefer_shared(pair_ws_kernel<FixedI, false, true>);
  prefer_shared(pair_ws_kernel<FixedI, true, true>);
  prefer_shared(pair_ws_kernel<Fp64, false, true>);
  prefer_shared(pair_ws_kernel<Fp64, true, true>);
  prefer_shared(adj_ws_kernel<FixedI, false>);
  prefer_shared(adj_ws_kernel<FixedI, true>);
  prefer_shared(adj_ws_kernel<Fp64, false>);
  prefer_shared(adj_ws_kernel<Fp64, true>);
  prefer_shared(adj2_kernel<FixedI, false>);
  prefer_shared(adj2_kernel<FixedI, true>);
  prefer_shared(adj2_kernel<Fp64, false>);
  prefer_shared(adj2_kernel<Fp64, true>);
}

template <bool ASYNC>
static void launch_fwd_stage_t(int arith, bool record, const FwdArgs& a, int grid,
                               cudaStream_t s) {
  if (arith == 1) {
    if (record)
      fwd_stage_kernel<Fixed, true, ASYNC><<<grid, NT, 0, s>>>(a);
    else
      fwd_stage_kernel<Fixed, false, ASYNC><<<grid, NT, 0, s>>>(a);
  } else {
    if (record)
      fwd_stage_kernel<Fp64, true, ASYNC><<<grid, NT, 0, s>>>(a);
    else
      fwd_stage_kernel<Fp64, false, ASYNC><<<grid, NT, 0, s>>>(a);
  }
}

cudaError_t launch_fwd_stage(int arith, bool record, int staging, const FwdArgs& a, int grid,
                             cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  set_carveouts();
  grid = min(grid, a.nitems);
  if (staging == 1)
    launch_fwd_stage_t<true>(arith, record, a, grid, s);
  else
    launch_fwd_stage_t<false>(arith, record, a, grid, s);
  return cudaGetLastError();
}

cudaError_t launch_lap(int arith, const LapArgs& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  set_carveouts();
  grid = min(grid, a.nitems);
  if (arith == 1)
    lap_kernel<Fixed><<<grid, NT, 0, s>>>(a);
  else
    lap_kernel<Fp64><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adj2(bool second, int arith, const Adj2Args& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  set_carveouts();
  grid = min(grid, a.nitems);
  if (arith == 1) {
    if (second)
      adj2_kernel<FixedI, true><<<grid, NT, 0, s>>>(a);
    else
      adj2_kernel<FixedI, false><<<grid, NT, 0, s>>>(a);
  } else {
    if (second)
      adj2_kernel<Fp64, true><<<grid, NT, 0, s>>>(a);
    else
      adj2_kernel<Fp64, false><<<grid, NT, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_combine(int arith, const DRect* rects, const DChunk* chunks,
                               int nchunks, const AdjCombineArgs& a, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  (void)grid;
  if (arith == 1)
    adj_combine_kernel<true><<<nchunks, kGatherChunk, 0, s>>>(rects, chunks, nchunks, a);
  else
    adj_combine_kernel<false><<<nchunks, kGatherChunk, 0, s>>>(rects, chunks, nchunks, a);
  return cudaGetLastError();
}

cudaError_t launch_pair(int arith, bool second, const PairArgs& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  set_carveouts();
  grid = min(grid, a.nitems);
  const bool rec = a.rec0 != nullptr;
  if (arith == 1) {
    if (second)
      rec ? pair_kernel<FixedI, true, true><<<grid, NT, 0, s>>>(a)
          : pair_kernel<FixedI, true, false><<<grid, NT, 0, s>>>(a);
    else
      rec ? pair_kernel<FixedI, false, true><<<grid, NT, 0, s>>>(a)
          : pair_kernel<FixedI, false, false><<<grid, NT, 0, s>>>(a);
  } else {
    if (second)
      rec ? pair_kernel<Fp64, true, true><<<grid, NT, 0, s>>>(a)
          : pair_kernel<Fp64, true, false><<<grid, NT, 0, s>>>(a);
    else
      rec ? pair_kernel<Fp64, false, true><<<grid, NT, 0, s>>>(a)
          : pair_kernel<Fp64, false, false><<<grid, NT, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// The warp-specialised kernels split the registers they were launched with
// between the roles (setmaxnreg); a launch with another count would leave the
// producers' increase waiting.  Checked once per kernel before its first launch.
template <class K>
static bool ws_regs_ok(K kernel) {
  cudaFuncAttributes at{};
  return cudaFuncGetAttributes(&at, kernel) == cudaSuccess && at.numRegs == kWsLaunchRegs &&
         at.maxThreadsPerBlock >= kWsThreads;
}
static bool ws_kernels_ok() {
  static const bool ok =
      ws_regs_ok(pair_ws_kernel<FixedI, false, false>) &&
      ws_regs_ok(pair_ws_kernel<FixedI, true, false>) &&
      ws_regs_ok(pair_ws_kernel<FixedI, false, true>) &&
      ws_regs_ok(pair_ws_kernel<FixedI, true, true>) &&
      ws_regs_ok(pair_ws_kernel<Fp64, false, false>) && ws_regs_ok(pair_ws_kernel<Fp64, true, false>) &&
      ws_regs_ok(pair_ws_kernel<Fp64, false, true>) && ws_regs_ok(pair_ws_kernel<Fp64, true, true>) &&
      ws_regs_ok(adj_ws_kernel<FixedI, false>) && ws_regs_ok(adj_ws_kernel<FixedI, true>) &&
      ws_regs_ok(adj_ws_kernel<Fp64, false>) && ws_regs_ok(adj_ws_kernel<Fp64, true>);
  return ok;
}

cudaError_t launch_pair_ws(int arith, bool second, const PairArgs& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  if (!ws_kernels_ok()) return cudaErrorInvalidConfiguration;
  set_carveouts();
  grid = min(grid, a.nitems);
  const bool rec = a.rec0 != nullptr;
  if (arith == 1) {
    if (second)
      rec ? pair_ws_kernel<FixedI, true, true><<<grid, kWsThreads, 0, s>>>(a)
          : pair_ws_kernel<FixedI, true, false><<<grid, kWsThreads, 0, s>>>(a);
    else
      rec ? pair_ws_kernel<FixedI, false, true><<<grid, kWsThreads, 0, s>>>(a)
          : pair_ws_kernel<FixedI, false, false><<<grid, kWsThreads, 0, s>>>(a);
  } else {
    if (second)
      rec ? pair_ws_kernel<Fp64, true, true><<<grid, kWsThreads, 0, s>>>(a)
          : pair_ws_kernel<Fp64, true, false><<<grid, kWsThreads, 0, s>>>(a);
    else
      rec ? pair_ws_kernel<Fp64, false, true><<<grid, kWsThreads, 0, s>>>(a)
          : pair_ws_kernel<Fp64, false, false><<<grid, kWsThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_ws(bool second, int arith, const AdjWsArgs& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  if (!ws_kernels_ok()) return cudaErrorInvalidConfiguration;
  set_carveouts();
  grid = min(grid, a.nitems);
  if (arith == 1) {
    if (second)
      adj_ws_kernel<FixedI, true><<<grid, kWsThreads, 0, s>>>(a);
    else
      adj_ws_kernel<FixedI, false><<<grid, kWsThreads, 0, s>>>(a);
  } else {
    if (second)
      adj_ws_kernel<Fp64, true><<<grid, kWsThreads, 0, s>>>(a);
    else
      adj_ws_kernel<Fp64, false><<<grid, kWsThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t pair_ws_occupancy(int arith, int* blocks_per_sm) {
  set_carveouts();
  if (arith == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, pair_ws_kernel<FixedI, true, true>, kWsThreads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, pair_ws_kernel<Fp64, true, true>, kWsThreads, 0);
}

cudaError_t pair_occupancy(int arith, int* blocks_per_sm) {
  set_carveouts();
  if (arith == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                         pair_kernel<FixedI, true, true>, NT, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                       pair_kernel<Fp64, true, true>, NT, 0);
}

cudaError_t launch_xfer(bool pack, const DXfer* xs, const DChunk* chunks, int nchunks,
                        double* f, double* g, double* buf, unsigned* emax, int ndom, int grid,
                        cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  grid = min(grid, nchunks);
  if (pack)
    xfer_kernel<true><<<grid, kGatherChunk, 0, s>>>(xs, chunks, nchunks, f, g, buf, nullptr, ndom);
  else
    xfer_kernel<false><<<grid, kGatherChunk, 0, s>>>(xs, chunks, nchunks, f, g, buf, emax, ndom);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const DProl* rects, const DChunk* chunks, int nchunks,
                           const double* du, const double* dp, double* fu, double* fp,
                           unsigned* emax, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  prolong_kernel<<<nchunks, 256, 0, s>>>(rects, chunks, nchunks, du, dp, fu, fp, emax);
  return cudaGetLastError();
}

cudaError_t launch_blend(const DRect* rects, const DChunk* chunks, int nchunks, const double* a0,
                         const double* a1, const double* b0, const double* b1, double alpha,
                         double* ao, double* bo, int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  blend_kernel<<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, a0, a1, b0, b1, alpha,
                                                  ao, bo);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const DRestr* rects, const DChunk* chunks, int nchunks,
                            const double* fu, const double* fp, double* cu, double* cp,
                            unsigned* emax, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  restrict_kernel<<<nchunks, kGatherChunk, 0, s>>>(rects, chunks, nchunks, fu, fp, cu, cp,
                                                   emax);
  return cudaGetLastError();
}

int stage_threads() { return NT; }

cudaError_t stage_occupancy(int arith, int staging, int* blocks_per_sm) {
  set_carveouts();
  if (staging == 1)
    return arith == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            blocks_per_sm, fwd_stage_kernel<Fixed, false, true>, NT, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            blocks_per_sm, fwd_stage_kernel<Fp64, false, true>, NT, 0);
  return arith == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          blocks_per_sm, fwd_stage_kernel<Fixed, false, false>, NT, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          blocks_per_sm, fwd_stage_kernel<Fp64, false, false>, NT, 0);
}

}  // namespace dev
}  // namespace sc
