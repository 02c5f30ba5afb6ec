// Kernel argument blocks and launchers (host/device shared declarations).
#pragma once

#include <cuda_runtime.h>

namespace sc {
namespace dev {

struct DBox;
struct DItem;
struct DRect;
struct DChunk;

// Per (stage, domain) coefficients of the nested RK4 form.
struct StageCoef {
  double gamma;    // g_s = c_s * dt, c = (1/4, 1/3, 1/2, 1)
  double kappa;    // g_s / (12 h^2)
  double inv12h2;  // 1 / (12 h^2)
  double pad;
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
  const StageCoef* coef;  // [ndom] of this stage
  const unsigned* emax_in;
  unsigned* emax_out;
  unsigned* emax_clear;
  unsigned* err;
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

struct AdjArgs {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* z_in;   // c2 * lam_s.pi (ghosts filled)
  const double* lam_u;  // lam_s.u
  const double* c2;
  double* lam_out;      // lam_{s-1}.u
  double* z_out;        // z_{s-1}
  const StageCoef* coef;  // [ndom] of stage s
  const unsigned* emax_in;
  unsigned* emax_out;
  unsigned* emax_clear;
  unsigned* err;
};

struct AdjLastArgs {
  const DItem* items;
  int nitems;
  int ndom;
  const DBox* boxes;
  const double* z_in;  // z_1
  const double* l1;    // lam_1.u
  const double* l2;    // lam_2.u
  const double* l3;    // lam_3.u
  double* yu;          // in: lam_4 = adjoint of the step output; out: of its input
  double* yp;
  const double* c2;
  const double* lapw1;  // recorded L w_0.u .. L w_3.u of the forward step
  const double* lapw2;
  const double* lapw3;
  const double* lapw4;
  double* c2bar;
  double* z_out;  // c2 * ybar.pi, first stencil input of the previous step
  const StageCoef* coef;  // [4 * ndom]
  const unsigned* emax_in;
  unsigned* emax_out;
  unsigned* emax_clear;
  unsigned* err;
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
cudaError_t launch_fwd_stage(int arith, bool record, const FwdArgs& a, int grid,
                             cudaStream_t s);
cudaError_t launch_lap(int arith, const LapArgs& a, int grid, cudaStream_t s);
cudaError_t launch_adj_stage(int arith, const AdjArgs& a, int grid, cudaStream_t s);
cudaError_t launch_adj_last(int arith, const AdjLastArgs& a, int grid, cudaStream_t s);
int stage_threads();
cudaError_t stage_occupancy(int arith, int* blocks_per_sm);

}  // namespace dev
}  // namespace sc
