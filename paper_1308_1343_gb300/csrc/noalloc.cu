// RK4 steps of one periodic box with library-static scratch memory.
//
// Some callers cannot allocate device memory: code that runs while a custom
// allocator owns the whole device, or an application that forbids
// cudaMalloc/cudaFree after start-up.  They can still advance a single
// periodic box with sc_box_rk4_step_noalloc: the four stage arrays the step
// needs live in one file-scope __device__ array of fixed size that the CUDA
// module itself provides, so the call makes no cudaMalloc, cudaFree or other
// allocating call.  The price is that every GPU that loads the library holds
// the array (kNoAllocScratchBytes) until the process exits.
//
// The arithmetic is the FP64 form of the level library's stage kernel (the
// same tile traversal, stencil sum and nested RK4 stages), so results agree
// with sc_level_rk4_step in SC_ARITH_FP64 with one stage per pass on a one-box
// periodic level.
#include <mutex>

#include "../../include/sc_level.h"
#include "kernels.cuh"
#include "level.hpp"

namespace sc {
namespace {

// Largest padded field (doubles) the static scratch holds, per stage array.
constexpr long long kNoAllocField = 1ll << 19;  // 4 MiB per array
constexpr long long kNoAllocScratchBytes = 4 * kNoAllocField * 8;  // 16 MiB in total

// The scratch: Wa.u, Wa.pi, Wb.u, Wb.pi, one after the other.
static __device__ __align__(256) double g_noalloc_scratch[4 * kNoAllocField];

constexpr int kNT = 256;
constexpr int kMaxDevices = 64;

// Device address of g_noalloc_scratch on each device, resolved once (host side
// the symbol is only a stand-in and must never be passed to a kernel).
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Fill the star ghosts of one periodic box by wrapping each ghost point onto
// the interior (the exchange list of a one-box periodic level, computed in
// place instead of read from a descriptor array).
__global__ void __launch_bounds__(256) noalloc_fill_kernel(double* f, dev::DBox bx) {
  const long long nx = bx.nx, ny = bx.ny, nz = bx.nz;
  const long long sx = 2 * ny * nz, sy = 2 * nx * nz, sz = 2 * nx * ny;  // per side
  const long long total = 2 * (sx + sy + sz);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long j = i;
    int axis = 0;
    long long side_n = sx;
    if (j >= 2 * sx) {
      j -= 2 * sx;
      axis = 1;
      side_n = sy;
      if (j >= 2 * sy) {
        j -= 2 * sy;
        axis = 2;
        side_n = sz;
      }
    }
    const int side = j >= side_n ? 1 : 0;
    if (side) j -= side_n;
    long long p[3];
    if (axis == 0) {  // j over (2, ny, nz), x fastest
      p[0] = j % 2; p[1] = (j / 2) % ny; p[2] = j / (2 * ny);
      p[0] = side ? nx + p[0] : p[0] - 2;
    } else if (axis == 1) {  // (nx, 2, nz)
      p[0] = j % nx; p[1] = (j / nx) % 2; p[2] = j / (2 * nx);
      p[1] = side ? ny + p[1] : p[1] - 2;
    } else {  // (nx, ny, 2)
      p[0] = j % nx; p[1] = (j / nx) % ny; p[2] = j / (nx * ny);
      p[2] = side ? nz + p[2] : p[2] - 2;
    }
    const long long q0 = (p[0] + nx) % nx, q1 = (p[1] + ny) % ny, q2 = (p[2] + nz) % nz;
    f[bx.off + p[0] + p[1] * bx.py + p[2] * bx.pz] = f[bx.off + q0 + q1 * bx.py + q2 * bx.pz];
  }
}

struct NoAllocEpi {
  static constexpr int NF = 4;  // w_in.pi, y.u, y.pi, c2
  const double* f[NF];
  double* wu_out;
  double* wp_out;
  double g, kap;
  __device__ __forceinline__ void point(int i, const double2* pw, double rA, double rB,
                                        bool actB, int, int, int) {
    const double2 wp = pw[0], u0 = pw[1], p0 = pw[2], c = pw[3];
    double2 un, pn;
    un.x = fma(g, wp.x, u0.x);
    un.y = fma(g, wp.y, u0.y);
    pn.x = fma(kap, c.x * rA, p0.x);
    pn.y = fma(kap, c.y * rB, p0.y);
    if (actB) {
      dev::st2(wu_out + i, un);
      dev::st2(wp_out + i, pn);
    } else {
      wu_out[i] = un.x;
      wp_out[i] = pn.x;
    }
  }
};

// One nested-RK4 stage over the box; work items are derived from the block
// index instead of being read from a list.
__global__ void __launch_bounds__(kNT, 4) noalloc_stage_kernel(
    dev::DBox bx, int txh, int tz, const double* wu_in, const double* wp_in, const double* yu,
    const double* yp, const double* c2, double* wu_out, double* wp_out, double g, double kap) {
  __shared__ dev::Smem<kNT, dev::Fp64, 4> smem;
  const int tx = 2 * txh, ty = kNT / txh;
  const int ntx = (bx.nx + tx - 1) / tx, nty = (bx.ny + ty - 1) / ty, ntz = (bx.nz + tz - 1) / tz;
  const int nitems = ntx * nty * ntz;
  unsigned err = 0;
  for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
    const int ix = i % ntx, iy = (i / ntx) % nty, iz = i / (ntx * nty);
    dev::DItem it{0, ix * tx, iy * ty, iz * tz, min(tz, bx.nz - iz * tz), txh};
    NoAllocEpi epi{{wp_in, yu, yp, c2}, wu_out, wp_out, g, kap};
    dev::run_item<kNT>(it, bx, wu_in, dev::Fp64{}, smem, err, epi);
  }
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace sc

using namespace sc;

// Messages below stay within the short-string buffer, so reporting an error
// allocates nothing either.
extern "C" int sc_box_rk4_step_noalloc(double* u, double* pi, const double* c2, int32_t nx,
                                       int32_t ny, int32_t nz, double h, double dt,
                                       int32_t nsteps, void* stream) {
  if (!aligned16(u) || !aligned16(pi) || !aligned16(c2)) return set_error(SC_EINVAL, "bad pointer");
  if (nx < 2 || ny < 2 || nz < 2 || nsteps < 0 || !(h > 0.0) || !(dt >= 0.0))
    return set_error(SC_EINVAL, "bad argument");
  // every extent fits the scratch on its own before any product is formed,
  // and the padded size is computed in 64 bits: no extent can wrap it
  if ((long long)nx > kNoAllocField || (long long)ny > kNoAllocField ||
      (long long)nz > kNoAllocField)
    return set_error(SC_EINVAL, "box too large");
  const long long py = ((long long)nx + 4 + 15) / 16 * 16;
  const long long pz = py * ((long long)ny + 4);
  if (pz > kNoAllocField || pz * ((long long)nz + 4) > kNoAllocField)
    return set_error(SC_EINVAL, "box too large");
  // an error left pending by earlier work belongs to that work: report it
  // as such instead of enqueuing more launches behind it
  if (cudaPeekAtLastError() != cudaSuccess) return set_error(SC_ECUDA, "earlier CUDA error pending");
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return set_error(SC_ECUDA, "no device");
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[device]) {
      double* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
      if (e != cudaSuccess || !p) return set_error(SC_ECUDA, "symbol address");
      g_scratch_addr[device] = p;
    }
    base = g_scratch_addr[device];
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return set_error(SC_ECUDA, "device query");
  const cudaStream_t s = (cudaStream_t)stream;
  dev::DBox bx{2 + 2 * py + 2 * pz, py, pz, nx, ny, nz, 0};
  const int txh = nx <= 16 ? 8 : (nx <= 32 ? 16 : 32);
  const int tz = 32;
  double* W[4] = {base, base + kNoAllocField, base + 2 * kNoAllocField, base + 3 * kNoAllocField};
  static const double c[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  double* in_u[4] = {u, W[0], W[2], W[0]};
  double* in_p[4] = {pi, W[1], W[3], W[1]};
  double* out_u[4] = {W[0], W[2], W[0], u};
  double* out_p[4] = {W[1], W[3], W[1], pi};
  for (int n = 0; n < nsteps; ++n)
    for (int st = 0; st < 4; ++st) {
      const double g = c[st] * dt;
      noalloc_fill_kernel<<<sms * 4, 256, 0, s>>>(in_u[st], bx);
      noalloc_stage_kernel<<<sms * 2, kNT, 0, s>>>(bx, txh, tz, in_u[st], in_p[st], u, pi, c2,
                                                    out_u[st], out_p[st], g,
                                                    g / (12.0 * h * h));
      // stop at the first launch that fails
      if (cudaGetLastError() != cudaSuccess) return set_error(SC_ECUDA, "launch failed");
    }
  return SC_OK;
}
