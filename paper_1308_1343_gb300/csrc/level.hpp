// Internal host-side representation of a level (not part of the C ABI).
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sc_level.h"
#include "descriptors.hpp"
#include "launch.hpp"

struct sc_level;

namespace sc {

int set_error(int code, const std::string& msg);
int ensure_device(sc_level* L);
int get_field(sc_level* L, const std::string& name, double** p);
int set_coef(sc_level* L, const double* dt, int ndt, cudaStream_t s);
int scratch4(sc_level* L, double* W[6]);
int upload_items(sc_level* L);
// DBox::wrap of box b: bit 0 the box alone tiles a domain periodic on every
// axis (x extent even, x and y extents >= 2), bit 1 also z extent >= 2
int wrap_bits(const sc_level* L, int b);
// Host plan of the x-face ghost copies that the warp-specialised producers
// read from the boxes that own them (sc_level::xread, xfaces, xcuts); called
// when the level's layout and exchange list are built
void plan_xface_reads(sc_level* L);
// Append the work items of box b (interior nx x ny x nz) for a tile of
// tx x ty points and z-runs of at most tz planes, z-major: the z extent is
// cut into ceil(nz / tz) runs whose lengths differ by at most one plane.
// the order of the batched launches' item list: by the place of the tile in
// its domain (domain, z, y, x of its first point)
void order_items(const sc_level* L, std::vector<dev::DItem>& items);
void append_box_items(std::vector<dev::DItem>& items, int b, int nx, int ny, int nz, int tx,
                      int ty, int tz, const std::vector<int>* cut_lo = nullptr,
                      const std::vector<int>* cut_hi = nullptr);
// nsteps RK4 steps as sc_level_rk4_step; qprep = false reuses the pre-scaled
// wave speeds of the previous call (same c2 and dt); bounds = true reuses
// the exponent bounds of (u, pi) left by the previous call's last pass, which
// every write to u and pi since must have raised (two stages per pass, fixed
// arithmetic; otherwise they are computed)
int level_steps(sc_level* L, double* u, double* pi, const double* c2, double dt, int nsteps,
                int mode, cudaStream_t s, bool qprep, bool bounds = false);

// One peer of a rank-local part of a distributed level: the ghost copies
// this rank sends to it (source boxes local) and receives from it
// (destination boxes local), each in the order of the whole level's
// exchange list, so that both ends of a pair agree on the buffer layout.
struct PeerLists {
  int peer = -1;
  std::vector<sc_copy> send, recv;  // the local side's box index is local
  int64_t send_points = 0, recv_points = 0;
  int64_t send_offset = 0, recv_offset = 0;  // doubles into the 2-field buffers
};

struct SizeClass {
  std::array<int64_t, 3> ext;  // interior extent rounded up to a multiple of 8
  sc_tile tile;
  bool fixed = false;          // tile set by sc_level_set_tuning / autotune
  // the tile the autotuner found for the one-role two-stage kernels while the
  // level runs the warp-specialised ones: the adjoint's pass kernels (one-role
  // kernels over two stencil fields) use it
  sc_tile tile_one{};
  bool has_one = false;
};

// Device-side state, created lazily on the first call that takes a stream.
struct DeviceState {
  int device = -1;
  int sms = 0;
  std::string gpu_name;
  cudaStream_t capture = nullptr;

  dev::DBox* boxes = nullptr;
  // work items of the batched launches, ordered by the place of their tile
  // in its domain (domain, z, y, x of the tile's first point): the tiles
  // that run at the same time are neighbours also across box faces, so the
  // halos they read from other boxes are still in L2 (measured: 1 % on the
  // pass kernels of the uneven 64-box level; one box: the box-major order)
  dev::DItem* items = nullptr;
  int nitems = 0;
  // the same items box by box, for the launches of one box (per-box mode)
  dev::DItem* items_box = nullptr;
  std::vector<int> box_items;  // per-box item ranges [b], [b+1] of items_box
  // items of the adjoint's pass kernels: tiles tuned for one-role kernels
  // (SizeClass::tile_one), or NULL to use `items`
  dev::DItem* items_one = nullptr;
  int nitems_one = 0;

  // ghost exchange as rectangles + chunks (sorted by destination box)
  dev::DRect* grects = nullptr;
  dev::DChunk* gchunks = nullptr;
  int ngchunks = 0;
  std::vector<int> box_gchunks;
  // the chunks of the gather list that the one-role stencil kernels need:
  // every ghost of a box that is not self-periodic (DBox::wrap), the z ghosts
  // of one that is
  dev::DChunk* gchunks_nw = nullptr;
  int ngchunks_nw = 0;
  // those the warp-specialised kernels need: the same without the z ghosts
  // of self-periodic boxes of two planes or more, which they read from the
  // periodic images
  dev::DChunk* gchunks_nz = nullptr;
  int ngchunks_nz = 0;
  std::vector<int> box_gchunks_nz;  // per-box ranges [b], [b+1] of gchunks_nz
  // x-face ghost copies that the warp-specialised kernels read from their
  // owners (sc_level::xfaces, uploaded; not in gchunks_nz), per box and side
  dev::DXGhost* xg = nullptr;
  int* xg_ofs = nullptr;  // [2 nboxes + 1], NULL if there are none
  std::vector<char> box_wrap;
  // interior rectangles (one per box) + chunks
  dev::DRect* irects = nullptr;
  dev::DChunk* ichunks = nullptr;
  int nichunks = 0;
  dev::DChunk* pchunks = nullptr;  // interior, kGatherChunk points per chunk
  int npchunks = 0;
  dev::DPush* push = nullptr;      // ghost copies grouped by source box and face slab
  int* push_gofs = nullptr;        // [6 nboxes + 1]
  // interior + the six ghost slabs of every box (all points the stencil reads)
  dev::DRect* srects = nullptr;
  dev::DChunk* schunks = nullptr;
  int nschunks = 0;

  dev::StageCoef* coef = nullptr;  // [4][ndom]
  dev::AdjCoef* acoef = nullptr;   // [ndom]
  std::vector<double> coef_dt;     // dt per domain the coefficients were built for
  double* inv12h2 = nullptr;       // [ndom]
  double* qfac = nullptr;          // [ndom][2]: dt/(12 h^2), (dt/3)/(12 h^2)
  double* h3 = nullptr;            // [ndom]
  unsigned* emax = nullptr;        // forward ring [4][ndom]
  unsigned* emax_adj = nullptr;    // adjoint slots [8][ndom]
  unsigned* err = nullptr;
  double* partial = nullptr;       // [nichunks]
  double* pinned = nullptr;        // host staging for small uploads
  size_t pinned_size = 0;

  // scratch fields, library-owned
  std::map<std::string, double*> fields;
  std::map<std::string, size_t> field_count;

  // distributed level: pack and unpack rectangles of every peer, in peer
  // order (DXfer, one per ghost copy that crosses ranks) and their chunks
  dev::DXfer* xsend = nullptr;
  dev::DChunk* xsend_chunks = nullptr;
  int nxsend_chunks = 0;
  dev::DXfer* xrecv = nullptr;
  dev::DChunk* xrecv_chunks = nullptr;
  int nxrecv_chunks = 0;

  // captured RK4 step graphs keyed by (u, pi, c2, arith, version)
  std::map<std::tuple<const void*, const void*, const void*, int, int>,
           std::pair<cudaGraphExec_t, int>>
      graphs;
  // per-kernel CUDA-event timing (mode SC_MODE_TIMED): kind -> event pairs
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_kind;  // SC_KERNEL_* of each timed launch
  int grid_stage = 0;  // persistent grid of the stage kernels
  int grid_stage_s[2] = {0, 0};  // of the one-stage kernel per staging
  int grid_pair = 0;   // persistent grid of the two-stage kernels
  int grid_pair_ws = 0;  // ... of their warp-specialised form
  int grid_small = 0;  // grid of the gather / reduction kernels
};

}  // namespace sc

struct sc_level {
  std::vector<sc_box> boxes;
  std::vector<sc_domain> doms;
  std::vector<int64_t> off, py, pz, storage;
  int64_t field_size = 0;
  std::vector<sc_copy> copies;
  // x-face ghost copies that the warp-specialised producers read from the
  // boxes that own them instead of having them gathered (plan_xface_reads):
  // per copy whether it is one; per box and side (2 b + side) those copies
  // as the kernels look them up; and per box and side the planes where their
  // z ranges start or end inside the box: work items at that x face end
  // their z-run there, so that each thread of an item reads its ghosts from
  // one box (measured: 1.6 % on the uneven level's pass kernels, where a
  // switch of source inside the plane loop cost 5 % there and 2 % on levels
  // without such ghosts)
  std::vector<char> xread;
  std::vector<std::vector<sc::dev::DXGhost>> xfaces;
  std::vector<std::vector<int>> xcuts;
  std::vector<int> box_class;
  std::vector<sc::SizeClass> classes;
  int arith = SC_ARITH_FIXED;
  int fuse = 2;             // RK4 stages per stencil pass of sc_level_rk4_step: 1 or 2
  bool fuse_fixed = false;  // set by sc_level_set_fusion; else the autotuner chooses
  int staging = 0;             // one-stage kernel: raw values in registers (0) or
                               // in shared memory by cp.async (1)
  bool staging_fixed = false;  // set by sc_level_set_staging; else the autotuner chooses
  int ctas_per_sm = 0;
  int pass_ws = 1;          // two-stage passes: one-role (0) or warp-specialised (1) kernels
  bool pass_fixed = false;  // set by sc_level_set_pass_kernel; else the autotuner chooses
  int wait_test = 0;        // failure-detection tests: the next warp-specialised pass
                            // launch withholds its ring slots (one shot)
  int version = 0;  // bumps when items change (invalidates graphs)
  int64_t launches = 0;
  int profile = 0;  // time every launch of the taped forward/backward
  bool all_periodic = true;
  // tape of the last sc_level_forward_tape
  bool tape_valid = false;
  int tape_nsteps = 0, tape_ckpt = 1;
  const double* tape_c2 = nullptr;
  std::vector<double> tape_dt;
  // rank-local part of a distributed level (sc_dist_create): only this
  // rank's boxes are stored; ghosts owned by other ranks' boxes arrive
  // through sc_dist_unpack
  bool partial = false;
  int rank = 0, nranks = 1;
  std::vector<int32_t> global_box;  // local box -> index in the whole level
  std::vector<sc::PeerLists> peers;  // by increasing peer rank
  int64_t send_doubles = 0, recv_doubles = 0;
  bool dist_begun = false;  // sc_dist_rk4_begin has started a run
  int dist_next_pass = 0;   // 0: pass A next, 1: pass B next
  const double* dist_u = nullptr;  // the run's state buffers
  const double* dist_pi = nullptr;
  sc::DeviceState* dev = nullptr;
};

namespace sc {

// Launch pass A (second == false) or B of the two-stage form with the level's
// pass kernel (one-role or warp-specialised); an armed wait test goes to this
// launch of the warp-specialised kernel and is then disarmed.
inline cudaError_t launch_pass(sc_level* L, bool second, dev::PairArgs a, cudaStream_t s) {
  if (!L->pass_ws) return dev::launch_pair(L->arith, second, a, L->dev->grid_pair, s);
  a.stall = L->wait_test;
  L->wait_test = 0;
  return dev::launch_pair_ws(L->arith, second, a, L->dev->grid_pair_ws, s);
}

}  // namespace sc
