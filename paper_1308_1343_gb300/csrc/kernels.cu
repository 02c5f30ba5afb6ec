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
// step).
#include "kernels.cuh"
#include "launch.hpp"

namespace sc {
namespace dev {

constexpr int NT = 256;

// ---------------------------------------------------------------------------
// Ghost gather: dst[ghost point] = src[owner point], every rectangle copy of
// the exchange list, one launch.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) gather_kernel(const DRect* __restrict__ rects,
                                                     const DChunk* __restrict__ chunks,
                                                     int nchunks, double* f) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const DChunk ch = chunks[c];
    const DRect r = rects[ch.rect];
    const int n = r.ex * r.ey * r.ez;
    const int end = min(ch.first + kChunk, n);
    for (int p = ch.first + threadIdx.x; p < end; p += blockDim.x) {
      const int x = p % r.ex;
      const int t = p / r.ex;
      const int y = t % r.ey;
      const int z = t / r.ey;
      f[r.dst + x + y * r.dpy + z * r.dpz] = f[r.src + x + y * r.spy + z * r.spz];
    }
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
  double g, lw;    // g_s; L w scale for recording
  unsigned emax;

  __device__ __forceinline__ void point(int i, const double2* pw, typename A::T rA,
                                        typename A::T rB, bool actB) {
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

template <class A, bool RECORD>
__global__ void __launch_bounds__(NT, 4) fwd_stage_kernel(FwdArgs a) {
  __shared__ Smem<NT, A, 4> smem;
  __shared__ unsigned red[NT / 32];
  if (A::kFixed) clear_slot(a.emax_clear, a.ndom);
  unsigned err = 0;
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const StageCoef cf = a.coef[bx.dom];
    const A arith = make_arith<A>(a.emax_in, bx.dom, err);
    FwdEpi<A, RECORD> epi{{a.wp_in, a.yu, a.yp, a.q}, a.wu_out, a.wp_out, a.lapw, arith,
                          a.qk, cf.gamma, cf.inv12h2 * exp2_int(-a.qk)};
    epi.emax = 0;
    run_item<NT>(it, bx, a.wu_in, arith, smem, err, epi);
    if (A::kFixed) cta_max_to(epi.emax, a.emax_out + bx.dom, red);
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
                                        typename A::T rB, bool actB) {
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
// Adjoint stages.  Reverse of w_s = y + g_s A w_{s-1} with
// A^T(a, b) = (L(c2 b), a), given lam_s (adjoint of w_s):
//   lam_{s-1}.u  = g_s L z_s,  z_s = c2 lam_s.pi
//   lam_{s-1}.pi = g_s lam_s.u
//   ybar        += lam_s            (and lam_0 at the end)
//   c2bar       += g_s lam_s.pi (L w_{s-1}.u)
// Stages s = 4, 3, 2 write lam_{s-1}.u and z_{s-1} = c2 g_s lam_s.u; the
// last kernel (s = 1) also forms ybar and c2bar from the stored lam_s.u and
// the recorded L w_{s-1}.u of the forward stages, and writes z_4 = c2 ybar.pi
// for the next (earlier) step.
// ---------------------------------------------------------------------------

template <class A>
struct AdjEpi {
  static constexpr int NF = 2;  // lam_s.u, c2
  const double* f[NF];
  double* __restrict__ lam_out;
  double* __restrict__ z_out;
  A arith;
  double g, kap;
  unsigned emax;
  __device__ __forceinline__ void point(int i, const double2* pw, typename A::T rA,
                                        typename A::T rB, bool actB) {
    const double2 l = pw[0], c = pw[1];
    const double2 lo = make_double2(kap * arith.scaled(rA, 0), kap * arith.scaled(rB, 0));
    const double2 zo = make_double2(c.x * (g * l.x), c.y * (g * l.y));
    if (actB) {
      st2(lam_out + i, lo);
      st2(z_out + i, zo);
    } else {
      lam_out[i] = lo.x;
      z_out[i] = zo.x;
    }
    if (A::kFixed) {
      emax = max(emax, biased_exp(zo.x));
      if (actB) emax = max(emax, biased_exp(zo.y));
    }
  }
};

template <class A>
__global__ void __launch_bounds__(NT, 4) adj_stage_kernel(AdjArgs a) {
  __shared__ Smem<NT, A, 2> smem;
  __shared__ unsigned red[NT / 32];
  if (A::kFixed) clear_slot(a.emax_clear, a.ndom);
  unsigned err = 0;
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const StageCoef cf = a.coef[bx.dom];
    const A arith = make_arith<A>(a.emax_in, bx.dom, err);
    AdjEpi<A> epi{{a.lam_u, a.c2}, a.lam_out, a.z_out, arith, cf.gamma, cf.kappa};
    epi.emax = 0;
    run_item<NT>(it, bx, a.z_in, arith, smem, err, epi);
    if (A::kFixed) cta_max_to(epi.emax, a.emax_out + bx.dom, red);
  }
  if (err) atomicOr(a.err, err);
}

template <class A>
struct AdjLastEpi {
  static constexpr int NF = 4;  // lam_1.u, lam_2.u, lam_3.u, lam_4.u (streamed)
  const double* f[NF];
  double* yu;
  double* yp;
  const double* __restrict__ c2;
  const double* __restrict__ w1;  // L w_0.u  (forward stage 1)
  const double* __restrict__ w2;
  const double* __restrict__ w3;
  const double* __restrict__ w4;  // L w_3.u  (forward stage 4)
  double* cb;
  double* __restrict__ z_out;
  A arith;
  double g1, g2, g3, g4, kap1;
  unsigned emax;
  __device__ __forceinline__ double pi_one(double p, double u, double b3, double b2,
                                           double b1) const {
    return p + fma(g4, u, fma(g3, b3, fma(g2, b2, g1 * b1)));
  }
  __device__ __forceinline__ double c2_one(double p, double u, double b3, double b2, double q4,
                                           double q3, double q2, double q1) const {
    // g4 lam4.pi Lw3 + g3 (g4 lam4.u) Lw2 + g2 (g3 lam3.u) Lw1 + g1 (g2 lam2.u) Lw0
    return fma(g4 * p, q4, fma(g3 * (g4 * u), q3, fma(g2 * (g3 * b3), q2, g1 * (g2 * b2) * q1)));
  }
  __device__ __forceinline__ void point(int i, const double2* pw, typename A::T rA,
                                        typename A::T rB, bool actB) {
    const double2 a1 = pw[0], a2 = pw[1], a3 = pw[2], u4 = pw[3];
    const double2 p4 = ld2(yp + i);
    const double2 l0 = make_double2(kap1 * arith.scaled(rA, 0), kap1 * arith.scaled(rB, 0));
    const double2 un = make_double2(((u4.x + a3.x) + (a2.x + a1.x)) + l0.x,
                                    ((u4.y + a3.y) + (a2.y + a1.y)) + l0.y);
    const double2 pn = make_double2(pi_one(p4.x, u4.x, a3.x, a2.x, a1.x),
                                    pi_one(p4.y, u4.y, a3.y, a2.y, a1.y));
    const double2 q4 = ld2(w4 + i), q3 = ld2(w3 + i), q2 = ld2(w2 + i), q1 = ld2(w1 + i);
    const double2 cbo = ld2(cb + i);
    const double2 cn = make_double2(
        cbo.x + c2_one(p4.x, u4.x, a3.x, a2.x, q4.x, q3.x, q2.x, q1.x),
        cbo.y + c2_one(p4.y, u4.y, a3.y, a2.y, q4.y, q3.y, q2.y, q1.y));
    const double2 cc = ld2(c2 + i);
    const double2 zo = make_double2(cc.x * pn.x, cc.y * pn.y);
    if (actB) {
      st2(yu + i, un);
      st2(yp + i, pn);
      st2(cb + i, cn);
      st2(z_out + i, zo);
    } else {
      yu[i] = un.x;
      yp[i] = pn.x;
      cb[i] = cn.x;
      z_out[i] = zo.x;
    }
    if (A::kFixed) {
      emax = max(emax, biased_exp(zo.x));
      if (actB) emax = max(emax, biased_exp(zo.y));
    }
  }
};

template <class A>
__global__ void __launch_bounds__(NT) adj_last_kernel(AdjLastArgs a) {
  __shared__ Smem<NT, A, 4> smem;
  __shared__ unsigned red[NT / 32];
  if (A::kFixed) clear_slot(a.emax_clear, a.ndom);
  unsigned err = 0;
  for (int i = blockIdx.x; i < a.nitems; i += gridDim.x) {
    const DItem it = a.items[i];
    const DBox bx = a.boxes[it.box];
    const A arith = make_arith<A>(a.emax_in, bx.dom, err);
    const int d = bx.dom, nd = a.ndom;
    AdjLastEpi<A> epi{{a.l1, a.l2, a.l3, a.yu}, a.yu, a.yp, a.c2, a.lapw1, a.lapw2,
                      a.lapw3, a.lapw4, a.c2bar, a.z_out, arith,
                              a.coef[0 * nd + d].gamma, a.coef[1 * nd + d].gamma,
                              a.coef[2 * nd + d].gamma, a.coef[3 * nd + d].gamma,
                      a.coef[0 * nd + d].kappa};
    epi.emax = 0;
    run_item<NT>(it, bx, a.z_in, arith, smem, err, epi);
    if (A::kFixed) cta_max_to(epi.emax, a.emax_out + bx.dom, red);
  }
  if (err) atomicOr(a.err, err);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

cudaError_t launch_gather(const DRect* rects, const DChunk* chunks, int nchunks, double* f,
                          int grid, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  gather_kernel<<<min(grid, nchunks), 256, 0, s>>>(rects, chunks, nchunks, f);
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

// Four 46 KB CTAs per SM need the largest shared-memory carveout.
template <class K>
void prefer_shared(K kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

static void set_carveouts() {
  static bool done = false;
  if (done) return;
  done = true;
  prefer_shared(fwd_stage_kernel<Fixed, true>);
  prefer_shared(fwd_stage_kernel<Fixed, false>);
  prefer_shared(fwd_stage_kernel<Fp64, true>);
  prefer_shared(fwd_stage_kernel<Fp64, false>);
  prefer_shared(adj_stage_kernel<Fixed>);
  prefer_shared(adj_stage_kernel<Fp64>);
  prefer_shared(adj_last_kernel<Fixed>);
  prefer_shared(adj_last_kernel<Fp64>);
  prefer_shared(lap_kernel<Fixed>);
  prefer_shared(lap_kernel<Fp64>);
}

cudaError_t launch_fwd_stage(int arith, bool record, const FwdArgs& a, int grid,
                             cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  set_carveouts();
  grid = min(grid, a.nitems);
  if (arith == 1) {
    if (record)
      fwd_stage_kernel<Fixed, true><<<grid, NT, 0, s>>>(a);
    else
      fwd_stage_kernel<Fixed, false><<<grid, NT, 0, s>>>(a);
  } else {
    if (record)
      fwd_stage_kernel<Fp64, true><<<grid, NT, 0, s>>>(a);
    else
      fwd_stage_kernel<Fp64, false><<<grid, NT, 0, s>>>(a);
  }
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

cudaError_t launch_adj_stage(int arith, const AdjArgs& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  set_carveouts();
  grid = min(grid, a.nitems);
  if (arith == 1)
    adj_stage_kernel<Fixed><<<grid, NT, 0, s>>>(a);
  else
    adj_stage_kernel<Fp64><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adj_last(int arith, const AdjLastArgs& a, int grid, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  grid = min(grid, a.nitems);
  if (arith == 1)
    adj_last_kernel<Fixed><<<grid, NT, 0, s>>>(a);
  else
    adj_last_kernel<Fp64><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

int stage_threads() { return NT; }

cudaError_t stage_occupancy(int arith, int* blocks_per_sm) {
  set_carveouts();
  if (arith == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, fwd_stage_kernel<Fixed, false>, NT, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                       fwd_stage_kernel<Fp64, false>, NT, 0);
}

}  // namespace dev
}  // namespace sc
