// Kernel argument blocks and launchers (host/device shared declarations).
#pragma once

#include <cuda_runtime.h>

namespace sc {
namespace dev {

struct DBox;
struct DItem;
struct DRect;
struct DChunk;
struct DXfer;
struct DPush;
struct DXGhost;
struct DProl;
struct DRestr;

// Per (stage, domain) coefficients of the nested RK4 form.
struct StageCoef {
  double gamma;    // g_s = c_s * dt, c = (1/4, 1/3, 1/2, 1)
  double kappa;    // g_s / (12 h^2)
  double inv12h2;  // 1 / (12 h^2)
  double rec;      // recording scale: C_s 2^-qk_s / (12 h^2) (see kernels.cu)
};

// Per-domain constants of the adjoint combination (see kernels.cu).
struct AdjCoef {
  double cu[4];  // ybar.u coefficients of Phat4, Phat3, Phat2, Phat1
  double cp[4];  // ybar.pi coefficients of a, Phat4, Phat3, Phat2
};

struct FwdArgs {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* wu_in;  // stencil input (ghosts filled)
  const double* wp_in;
  const double* yu;
  const double* yp;
  const double* c2;
  double* wu_out;
  double* wp_out;
  double* lapw;  // recorded L w_in.u (adjoint checkpoints) or nullptr
  const double* q;  // c2 dt/(12 h^2) or c2 (dt/3)/(12 h^2), pre-scaled per run
  int qk;           // stage factor 2^qk on q
  const DPush* push;     // ghost copies grouped by source box and face slab
  const int* push_gofs;
  const StageCoef* coef;  // [ndom] of this stage
  const unsigned* emax_in;
  unsigned* emax_out;
  unsigned* emax_clear;
  unsigned* err;
};

// Two RK4 stages per pass (pass A: stages 1-2, pass B: stages 3-4).
struct PairArgs {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* s0;  // stencil fields, ghosts filled: A: y.u, y.pi.  B: w_2.u, w_2.pi
  const double* s1;
  const double* yu;  // pointwise: the step input y
  const double* yp;
  const double* q;   // c2 dt/(12 h^2), pre-scaled per run
  const double* x;   // A: c2 (dt/3)/(12 h^2).  B: 12 h^2 L y.u written by A
  double* out_u;     // A: w_2.u, w_2.pi.  B: y.u, y.pi (in place)
  double* out_p;
  double* ly;        // A: 12 h^2 L y.u
  double* rec0;      // or NULL; else C_s L w_{s-1}.u of the pass's two stages,
  double* rec1;      //   scaled as the stage kernel records them
  const StageCoef* coef;    // [4 ndom], stage s at s * ndom
  const unsigned* emax_in;  // [2 ndom]: exponent bounds of s0, s1
  unsigned* emax_out;       // [2 ndom]: of out_u, out_p (zero on entry)
  unsigned* err;
  int stall;                // warp-specialised kernels, failure-detection tests
                            // only: consumers never release a ring slot
  // warp-specialised kernels: x-face ghosts read from their owners, per box
  // and side entries [xg_ofs[2 b + side], xg_ofs[2 b + side + 1]) (or NULL)
  const DXGhost* xg;
  const int* xg_ofs;
};

struct LapArgs {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* u;
  double* out;
  const double* inv12h2;  // [ndom]
  const unsigned* emax_in;
  unsigned* err;
};

// Two applications of M = L(c2 .) per pass (see kernels.cu, adj2_kernel).
struct Adj2Args {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* z0_in;  // stencil inputs, ghosts filled
  const double* z1_in;
  const double* c2;
  double* p0_out;       // Phat = 12 h^2 L z_in
  double* p1_out;
  double* z0_out;       // first pass: c2 Phat, ghosts pushed
  double* z1_out;
  const DPush* push;
  const int* push_gofs;
  const unsigned* emax_in;  // [2 ndom]
  unsigned* emax_out;       // [2 ndom] (first pass)
  unsigned* emax_clear;     // [2 ndom] zeroed for a later launch, or NULL
  unsigned* err;
};

// The adjoint step in two warp-specialised passes (kernels.cu, adj_ws_kernel):
//   first : (Phat4, Phat3) = L^ (z0_in, z1_in) = L^ (c2 b, c2 a); writes
//           z0_out = c2 Phat4, z1_out = c2 Phat3 (stencil inputs of the second
//           pass), the parts of ybar that need Phat4 and Phat3 into yu, yp
//           (in place), and the whole c2bar update (in place);
//   second: (Phat2, Phat1) = L^ (z0_in, z1_in); completes ybar in yu, yp and
//           writes z0_out = c2 ybar.pi, z1_out = c2 ybar.u (the next adjoint
//           step's stencil inputs).
struct AdjWsArgs {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* z0_in;
  const double* z1_in;
  const double* c2;
  double* yu;
  double* yp;
  double* c2bar;      // first pass
  const double* q1;   // first pass: recorded C_1 Lw0 ... C_4 Lw3
  const double* q2;
  const double* q3;
  const double* q4;
  double* z0_out;
  double* z1_out;
  const AdjCoef* coef;      // [ndom]
  const unsigned* emax_in;  // [2 ndom]: bounds of z0_in, z1_in
  unsigned* emax_out;       // [2 ndom]: of z0_out, z1_out (zero on entry)
  unsigned* emax_clear;     // [2 ndom] zeroed by the kernel for a later launch
  unsigned* err;
  int stall;                // failure-detection tests only (as PairArgs)
  const DXGhost* xg;        // as PairArgs
  const int* xg_ofs;
};

struct AdjCombineArgs {
  double* yu;          // in: a (adjoint of the step output); out: of its input
  double* yp;          // in: b; out
  const double* p4;    // Phat4 .. Phat1
  const double* p3;
  const double* p2;
  const double* p1;
  const double* q1;    // recorded C_1 Lw0 ... C_4 Lw3 of the forward step
  const double* q2;
  const double* q3;
  const double* q4;
  const double* c2;
  double* c2bar;
  double* x_out;       // c2 ybar.pi: next adjoint step's first stencil input
  double* y_out;       // c2 ybar.u (both with ghosts pushed)
  const AdjCoef* coef; // [ndom]
  const DBox* boxes;
  const DPush* push;
  const int* push_gofs;
  unsigned* emax_x;
  unsigned* emax_y;
};

cudaError_t launch_gather(const DRect* rects, const DChunk* chunks, int nchunks, double* f,
                          int grid, cudaStream_t s);
cudaError_t launch_maxexp(const DRect* rects, const DChunk* chunks, int nchunks,
                          const double* f, unsigned* emax, unsigned* err, int grid,
                          cudaStream_t s);
cudaError_t launch_mul(const DRect* rects, const DChunk* chunks, int nchunks, const double* a,
                       const double* b, double* out, unsigned* emax, int grid,
                       cudaStream_t s);
cudaError_t launch_qprep(const DRect* rects, const DChunk* chunks, int nchunks,
                         const double* c2, double* qa, double* qb, const double* fac, int grid,
                         cudaStream_t s);
cudaError_t launch_misfit(const DRect* rects, const DChunk* chunks, int nchunks,
                          const double* u, const double* uo, double* seed, const double* h3,
                          double* partial, double* loss, int grid, cudaStream_t s);
// staging: 0 raw column and halo values in registers, 1 in shared memory by
// cp.async
cudaError_t launch_fwd_stage(int arith, bool record, int staging, const FwdArgs& a, int grid,
                             cudaStream_t s);
cudaError_t launch_lap(int arith, const LapArgs& a, int grid, cudaStream_t s);
cudaError_t launch_pair(int arith, bool second, const PairArgs& a, int grid, cudaStream_t s);
cudaError_t pair_occupancy(int arith, int* blocks_per_sm);
// the warp-specialised pass kernels (384 threads: 8 producer, 4 consumer warps)
cudaError_t launch_pair_ws(int arith, bool second, const PairArgs& a, int grid, cudaStream_t s);
cudaError_t pair_ws_occupancy(int arith, int* blocks_per_sm);
cudaError_t launch_adj_ws(bool second, int arith, const AdjWsArgs& a, int grid, cudaStream_t s);
// two fields over one exchange list; block 0 zeroes clear[0..nclear)
cudaError_t launch_gather2(const DRect* rects, const DChunk* chunks, int nchunks, double* f,
                           double* g, unsigned* clear, int nclear, cudaStream_t s);
cudaError_t launch_adj2(bool second, int arith, const Adj2Args& a, int grid, cudaStream_t s);
cudaError_t launch_adj_combine(int arith, const DRect* rects, const DChunk* chunks,
                               int nchunks, const AdjCombineArgs& a, int grid, cudaStream_t s);
// du, dp: the coarse data at the prolongation's time (see blend); emax (or
// NULL): the fine level's two exponent-bound slots of (u, pi), which take
// the largest biased exponent written (atomicMax)
cudaError_t launch_prolong(const DProl* rects, const DChunk* chunks, int nchunks,
                           const double* du, const double* dp, double* fu, double* fp,
                           unsigned* emax, cudaStream_t s);
// ao = (1 - alpha) a0 + alpha a1, bo likewise, on the rectangles
cudaError_t launch_blend(const DRect* rects, const DChunk* chunks, int nchunks, const double* a0,
                         const double* a1, const double* b0, const double* b1, double alpha,
                         double* ao, double* bo, int grid, cudaStream_t s);
// emax (or NULL): as for launch_prolong, the coarse level's slots
cudaError_t launch_restrict(const DRestr* rects, const DChunk* chunks, int nchunks,
                            const double* fu, const double* fp, double* cu, double* cp,
                            unsigned* emax, cudaStream_t s);
// distributed level: pack the rectangles of f and g into buf (pack), or
// write buf into them and raise emax[dom], emax[ndom + dom] (emax may be NULL)
cudaError_t launch_xfer(bool pack, const DXfer* xs, const DChunk* chunks, int nchunks,
                        double* f, double* g, double* buf, unsigned* emax, int ndom, int grid,
                        cudaStream_t s);
int stage_threads();
cudaError_t stage_occupancy(int arith, int staging, int* blocks_per_sm);

}  // namespace dev
}  // namespace sc
