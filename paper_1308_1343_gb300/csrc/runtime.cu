// Device side of the C ABI: descriptor upload, kernel enqueueing, the RK4
// step (per-box launches, batched launches, or a CUDA graph per step), the
// end-to-end host entry point, the misfit, and the checkpointed adjoint.
#include <algorithm>
#include <tuple>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sc_dist.h"
#include "level.hpp"

namespace sc {

using dev::DBox;
using dev::DChunk;
using dev::DItem;
using dev::DPush;
using dev::DXGhost;
using dev::DRect;
using dev::DXfer;
using dev::StageCoef;

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  return set_error(SC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SC_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <class T>
int upload(T** dst, const std::vector<T>& v) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (v.empty()) return SC_OK;
  SC_CUDA(cudaMalloc(dst, v.size() * sizeof(T)));
  SC_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SC_OK;
}

// Host check of a device list entry before upload: the elements of an
// ex x ey x ez rectangle with first element e0 and pitches (1, py, pz) (all
// non-negative) lie in a field of n elements.  A list built wrong fails
// here, on the host, instead of as an out-of-bounds access on the device.
bool rect_in_field(int64_t e0, int64_t py, int64_t pz, int64_t ex, int64_t ey, int64_t ez,
                   int64_t n) {
  if (ex <= 0 || ey <= 0 || ez <= 0) return true;
  return e0 >= 0 && e0 + (ex - 1) + (ey - 1) * py + (ez - 1) * pz < n;
}

int list_error(const char* what) {
  return set_error(SC_EINVAL, std::string("internal: a ") + what +
                                  " entry lies outside its field (please report)");
}

void add_chunks(int rect, int64_t n, std::vector<DChunk>& out, int chunk = dev::kChunk) {
  for (int64_t f = 0; f < n; f += chunk) out.push_back(DChunk{rect, (int)f});
}

// Work items: every box cut into (tile_x, tile_y, tile_z) items of its class,
// box-major, then z, y, x (one_role: the classes' tile_one instead).
void build_items(const sc_level* L, std::vector<DItem>& items, std::vector<int>& box_items,
                 bool one_role = false) {
  items.clear();
  box_items.assign(L->boxes.size() + 1, 0);
  for (size_t b = 0; b < L->boxes.size(); ++b) {
    box_items[b] = (int)items.size();
    const sc_box& B = L->boxes[b];
    const SizeClass& C = L->classes[L->box_class[b]];
    const sc_tile& t = one_role && C.has_one ? C.tile_one : C.tile;
    const auto& cuts = L->xcuts;
    const bool cut = cuts.size() == 2 * L->boxes.size();
    append_box_items(items, (int)b, (int)(B.hi[0] - B.lo[0]), (int)(B.hi[1] - B.lo[1]),
                     (int)(B.hi[2] - B.lo[2]), t.tile_x, t.tile_y, t.tile_z,
                     cut ? &cuts[2 * b] : nullptr, cut ? &cuts[2 * b + 1] : nullptr);
  }
  box_items[L->boxes.size()] = (int)items.size();
}

}  // namespace

int wrap_bits(const sc_level* L, int b) {
  // self-periodic: the box is its domain, periodic on every axis; the
  // kernels then read the owners of its x and y ghosts by wrapping the
  // coordinates (pairs of x-points stay 16-byte aligned for an even x
  // extent), the warp-specialised ones those of its z ghosts too (two
  // planes or more); the one-role kernels have its z ghosts gathered
  const sc_box& B = L->boxes[b];
  const sc_domain& Dm = L->doms[B.domain];
  bool self = Dm.periodic == 7u;
  for (int d = 0; d < 3; ++d) self = self && B.lo[d] == Dm.lo[d] && B.hi[d] == Dm.hi[d];
  self = self && B.hi[0] - B.lo[0] >= 2 && B.hi[1] - B.lo[1] >= 2 &&
         (B.hi[0] - B.lo[0]) % 2 == 0;
  if (!self) return 0;
  return 1 | (B.hi[2] - B.lo[2] >= 2 ? 2 : 0);
}

void plan_xface_reads(sc_level* L) {
  const int nb = (int)L->boxes.size();
  L->xread.assign(L->copies.size(), 0);
  L->xfaces.assign((size_t)2 * nb, {});
  L->xcuts.assign((size_t)2 * nb, {});
  auto index_of = [&](int b, const int64_t p[3]) {
    const sc_box& B = L->boxes[b];
    return L->off[b] + (p[0] - B.lo[0]) + (p[1] - B.lo[1]) * L->py[b] +
           (p[2] - B.lo[2]) * L->pz[b];
  };
  for (size_t c = 0; c < L->copies.size(); ++c) {
    const sc_copy& C = L->copies[c];
    const int b = C.dst_box;
    const sc_box& Bd = L->boxes[b];
    // a copy into the x-face ghost pair of a box of even x extent (not
    // self-periodic), 16-byte pairs at both ends, rows and planes inside
    // the box (x-face rows are the costly part of a gather: 16 bytes, half
    // of a 32-byte sector at both ends)
    const int side = C.dst_lo[0] == Bd.lo[0] - 2 ? 0 : (C.dst_lo[0] == Bd.hi[0] ? 1 : -1);
    const int64_t src = index_of(C.src_box, C.src_lo), dst = index_of(b, C.dst_lo);
    const bool xr = side >= 0 && C.ext[0] == 2 && src % 2 == 0 && dst % 2 == 0 &&
                    !wrap_bits(L, b) && (Bd.hi[0] - Bd.lo[0]) % 2 == 0 &&
                    C.dst_lo[1] >= Bd.lo[1] && C.dst_lo[1] + C.ext[1] <= Bd.hi[1] &&
                    C.dst_lo[2] >= Bd.lo[2] && C.dst_lo[2] + C.ext[2] <= Bd.hi[2];
    if (!xr) continue;
    L->xread[c] = 1;
    const int y0 = (int)(C.dst_lo[1] - Bd.lo[1]), z0 = (int)(C.dst_lo[2] - Bd.lo[2]);
    L->xfaces[(size_t)2 * b + side].push_back(
        dev::DXGhost{y0, y0 + (int)C.ext[1], z0, z0 + (int)C.ext[2], (int)src,
                     (int)L->py[C.src_box], (int)L->pz[C.src_box], C.src_box});
  }
  for (int g = 0; g < 2 * nb; ++g) {
    const int nz = (int)(L->boxes[g / 2].hi[2] - L->boxes[g / 2].lo[2]);
    auto& cuts = L->xcuts[g];
    for (const dev::DXGhost& e : L->xfaces[g])
      for (int z : {e.z0, e.z1})
        if (z > 0 && z < nz) cuts.push_back(z);
    std::sort(cuts.begin(), cuts.end());
    cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());
  }
}


void append_box_items(std::vector<DItem>& items, int b, int nx, int ny, int nz, int tx, int ty,
                      int tz, const std::vector<int>* cut_lo, const std::vector<int>* cut_hi) {
  // z-runs of at most tz planes, of balanced lengths, over [a, b)
  auto runs_of = [tz](int a, int b, std::vector<std::pair<int, int>>& out) {
    const int n = b - a, k = (n + tz - 1) / tz, base = n / k, extra = n % k;
    for (int r = 0, z = a; r < k; ++r) {
      const int len = base + (r < extra ? 1 : 0);
      out.emplace_back(z, len);
      z += len;
    }
  };
  std::vector<std::pair<int, int>> reg, edge[4];
  runs_of(0, nz, reg);
  // a column of tiles at an x face whose ghosts are read from their owners
  // splits [0, nz) where the owner changes first, then into runs: no run
  // crosses an owner change, and none is much shorter than it must be
  // (kind: 1 low face, 2 high face, 3 both)
  for (int kind = 1; kind < 4; ++kind) {
    std::vector<int> at{0, nz};
    for (const std::vector<int>* c : {kind & 1 ? cut_lo : nullptr, kind & 2 ? cut_hi : nullptr})
      if (c)
        for (int z : *c)
          if (z > 0 && z < nz) at.push_back(z);
    std::sort(at.begin(), at.end());
    at.erase(std::unique(at.begin(), at.end()), at.end());
    for (size_t i = 0; i + 1 < at.size(); ++i) runs_of(at[i], at[i + 1], edge[kind]);
  }
  // Tile columns: the class's width tx while a whole tile fits, then the
  // rest of the box's width in narrower tiles of the same thread count,
  // each tx * ty / w rows tall: either width halved while it does not fit,
  // down to 8 points (the last one may be ragged), or one tile of the
  // narrowest width that holds the rest, whichever takes fewer tiles over
  // the box's rows (the first, on a tie).  A remainder of 8 points under a
  // 32-wide tile would otherwise leave three quarters of the tile's threads
  // idle on every plane: on the 64-box uneven level a third of the tile
  // planes were ragged so.  (An 8 x 64 tile has the 64 x 8 tile's halo
  // buffer size, the largest the kernels hold.)
  std::vector<std::pair<int, int>> cols;  // (x0, width)
  const int xfull = nx / tx * tx;
  for (int x0 = 0; x0 < xfull; x0 += tx) cols.emplace_back(x0, tx);
  if (xfull < nx) {
    auto tiles_over_rows = [&](int w) { return (ny + ty * tx / w - 1) / (ty * tx / w); };
    std::vector<std::pair<int, int>> halved;
    int nh = 0;
    for (int x0 = xfull; x0 < nx;) {
      int w = tx;
      while (w > 8 && x0 + w > nx) w /= 2;
      halved.emplace_back(x0, w);
      nh += tiles_over_rows(w);
      x0 += w;
    }
    int w1 = 8;
    while (w1 < nx - xfull) w1 *= 2;
    if (tiles_over_rows(w1) < nh)
      cols.emplace_back(xfull, w1);
    else
      cols.insert(cols.end(), halved.begin(), halved.end());
  }
  // The last band of rows under the full-width columns, where it is at most
  // half a tile tall: wider, flatter tiles (height halved while the band
  // still fits, width doubled up to 64), each as wide as fits in the
  // columns' extent, down to the class's tile (ragged in y).
  const int fullRows = ny / ty * ty, band = ny - fullRows;
  int xm = 0;  // extent of the full-width columns
  for (const auto& c : cols)
    if (c.second == tx) xm = c.first + tx;
  int bh = ty, bw = tx;
  if (band > 0 && 2 * band <= ty && tx < 64 && xm > 0) {
    bh = ty / 2;
    bw = 2 * tx;
    while (bh / 2 >= band && bw < 64) {
      bh /= 2;
      bw *= 2;
    }
  }
  auto emit = [&](int x0, int w, int y0, int z0, int z1) {
    const int kind = (x0 == 0 && cut_lo && !cut_lo->empty() ? 1 : 0) |
                     (x0 + w >= nx && cut_hi && !cut_hi->empty() ? 2 : 0);
    if (!kind) {
      items.push_back(DItem{b, x0, y0, z0, z1 - z0, w / 2});
      return;
    }
    for (const auto& run : edge[kind])
      if (run.first >= z0 && run.first < z1)
        items.push_back(DItem{b, x0, y0, run.first, run.second, w / 2});
  };
  // run-major order: a column's runs that start inside regular run r go
  // with run r; the full-width tiles row by row, the band, then the
  // narrower columns
  for (size_t r = 0; r < reg.size(); ++r) {
    const int z0 = reg[r].first, z1 = z0 + reg[r].second;
    const int yEnd = bw != tx ? fullRows : ny;
    for (int y0 = 0; y0 < yEnd; y0 += ty)
      for (const auto& c : cols)
        if (c.second == tx) emit(c.first, tx, y0, z0, z1);
    if (bw != tx)
      for (int x0 = 0; x0 < xm;) {
        int w = bw;
        while (w > tx && x0 + w > xm) w /= 2;
        emit(x0, w, fullRows, z0, z1);
        x0 += w;
      }
    for (const auto& c : cols)
      if (c.second != tx)
        for (int y0 = 0; y0 < ny; y0 += ty * tx / c.second) emit(c.first, c.second, y0, z0, z1);
  }
}

void order_items(const sc_level* L, std::vector<DItem>& items) {
  auto key = [L](const DItem& it) {
    const sc_box& B = L->boxes[it.box];
    return std::make_tuple(B.domain, B.lo[2] + it.z0, B.lo[1] + it.y0, B.lo[0] + it.x0);
  };
  std::stable_sort(items.begin(), items.end(),
                   [&](const DItem& a, const DItem& b) { return key(a) < key(b); });
}

int upload_items(sc_level* L) {
  DeviceState* D = L->dev;
  for (int st = 0; st < 2; ++st) {
    int occ = 0;
    SC_CUDA(dev::stage_occupancy(L->arith, st, &occ));
    D->grid_stage_s[st] = D->sms * (L->ctas_per_sm > 0 ? L->ctas_per_sm : std::max(1, occ));
  }
  // register staging: also the grid of the Laplacian kernel
  D->grid_stage = D->grid_stage_s[0];
  int occ2 = 0, occ3 = 0;
  SC_CUDA(dev::pair_occupancy(L->arith, &occ2));
  D->grid_pair = D->sms * std::max(1, occ2);
  SC_CUDA(dev::pair_ws_occupancy(L->arith, &occ3));
  D->grid_pair_ws = D->sms * std::max(1, occ3);
  std::vector<DItem> items;
  build_items(L, items, D->box_items);
  // heuristic first choice (the paper's initial parameters, Sec. 3.2): while
  // the level's items do not fill two waves of the persistent grid, halve the
  // z-run of every class whose tile was not set explicitly
  for (;;) {
    if ((int)items.size() >= 2 * D->grid_stage) break;
    bool any = false;
    for (auto& c : L->classes)
      if (!c.fixed && c.tile.tile_z > 4) {
        c.tile.tile_z /= 2;
        any = true;
      }
    if (!any) break;
    build_items(L, items, D->box_items);
  }
  // the captured graphs name the old list: drop them first, so that a failed
  // upload leaves an empty list and no graph that reads freed memory
  SC_CUDA(cudaDeviceSynchronize());
  for (auto& kv : D->graphs) cudaGraphExecDestroy(kv.second.first);
  D->graphs.clear();
  L->version++;
  D->nitems = 0;
  int rc = upload(&D->items_box, items);
  if (rc) return rc;
  {
    std::vector<DItem> g = items;
    order_items(L, g);
    if ((rc = upload(&D->items, g))) return rc;
  }
  D->nitems = (int)items.size();
  // the adjoint's pass kernels: their own list where the tuner found other
  // tiles for one-role kernels
  bool other = false;
  for (const auto& c : L->classes)
    if (c.has_one && (c.tile_one.tile_x != c.tile.tile_x || c.tile_one.tile_z != c.tile.tile_z))
      other = true;
  D->nitems_one = 0;
  if (D->items_one) cudaFree(D->items_one);
  D->items_one = nullptr;
  if (other) {
    std::vector<DItem> one;
    std::vector<int> box_one;
    build_items(L, one, box_one, true);
    if ((rc = upload(&D->items_one, one))) return rc;
    D->nitems_one = (int)one.size();
  }
  return SC_OK;
}

void release_device(sc_level* L) {
  DeviceState* D = L->dev;
  if (!D) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != D->device) cudaSetDevice(D->device);
  cudaDeviceSynchronize();
  for (auto& kv : D->graphs) cudaGraphExecDestroy(kv.second.first);
  for (auto& pr : D->ev_pool) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto& kv : D->fields) cudaFree(kv.second);
  void* ptrs[] = {D->boxes, D->items, D->items_box, D->items_one, D->grects, D->gchunks, D->gchunks_nw,
                  D->gchunks_nz, D->xg, D->xg_ofs,
                  D->irects, D->ichunks,
                  D->srects, D->schunks, D->pchunks, D->push, D->push_gofs, D->coef, D->acoef, D->inv12h2, D->qfac, D->h3, D->emax,
                  D->emax_adj, D->err, D->partial, D->xsend, D->xsend_chunks, D->xrecv,
                  D->xrecv_chunks};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (D->pinned) cudaFreeHost(D->pinned);
  if (D->capture) cudaStreamDestroy(D->capture);
  if (cur != D->device && cur >= 0) cudaSetDevice(cur);
  delete D;
  L->dev = nullptr;
}

static int init_device(sc_level* L, int cur);

int ensure_device(sc_level* L) {
  int cur = -1;
  SC_CUDA(cudaGetDevice(&cur));
  if (L->dev) {
    if (L->dev->device != cur)
      return set_error(SC_EINVAL, "level was set up on another device");
    return SC_OK;
  }
  // a failed set-up leaves no partial device state behind: the next call
  // starts again from nothing (the error message of this one is kept)
  const int rc = init_device(L, cur);
  if (rc) {
    const std::string msg = sc_last_error();
    release_device(L);
    set_error(rc, msg);
  }
  return rc;
}

// Pack and unpack rectangles of a distributed level: one DXfer per ghost
// copy that crosses ranks, peer by peer in increasing rank, each copy's
// points at consecutive buffer positions from its peer's block offset (the
// buffer layout of include/sc_dist.h), chunked for one point per thread.
static int build_xfer_lists(sc_level* L) {
  DeviceState* D = L->dev;
  for (int dir = 0; dir < 2; ++dir) {  // 0: send (pack), 1: receive (unpack)
    std::vector<DXfer> xs;
    std::vector<DChunk> chunks;
    const int64_t total = dir ? L->recv_doubles : L->send_doubles;
    for (const PeerLists& P : L->peers) {
      const std::vector<sc_copy>& v = dir ? P.recv : P.send;
      const int64_t npts = dir ? P.recv_points : P.send_points;
      const int64_t start = dir ? P.recv_offset : P.send_offset;
      const int64_t end = start + npts;  // the first field's run of this peer
      if (start < 0 || start + 2 * npts > total) return list_error("exchange-buffer");
      int64_t pos = start;
      for (const sc_copy& C : v) {
        const int b = dir ? C.dst_box : C.src_box;
        const int64_t* lo = dir ? C.dst_lo : C.src_lo;
        const sc_box& B = L->boxes[b];
        DXfer x{};
        x.fld = L->off[b] + (lo[0] - B.lo[0]) + (lo[1] - B.lo[1]) * L->py[b] +
                (lo[2] - B.lo[2]) * L->pz[b];
        x.buf = pos;
        x.fpy = L->py[b];
        x.fpz = L->pz[b];
        x.ex = (int)C.ext[0];
        x.ey = (int)C.ext[1];
        x.ez = (int)C.ext[2];
        x.dom = B.domain;
        x.second = (int)npts;
        const int64_t n = C.ext[0] * C.ext[1] * C.ext[2];
        // the field rectangle lies in the field; its first-field run
        // [pos, pos + n) lies in the peer's first-field run [start, end),
        // so its second-field run (npts later) lies in [end, end + npts)
        if (!rect_in_field(x.fld, x.fpy, x.fpz, x.ex, x.ey, x.ez, L->field_size) ||
            pos + n > end)
          return list_error("exchange-buffer");
        pos += n;
        xs.push_back(x);
        add_chunks((int)xs.size() - 1, n, chunks, dev::kGatherChunk);
      }
      if (pos != end) return list_error("exchange-buffer");
    }
    int rc = upload(dir ? &D->xrecv : &D->xsend, xs);
    if (!rc) rc = upload(dir ? &D->xrecv_chunks : &D->xsend_chunks, chunks);
    if (rc) return rc;
    (dir ? D->nxrecv_chunks : D->nxsend_chunks) = (int)chunks.size();
  }
  return SC_OK;
}

static int init_device(sc_level* L, int cur) {
  DeviceState* D = new DeviceState();
  L->dev = D;
  D->device = cur;
  cudaDeviceProp p;
  SC_CUDA(cudaGetDeviceProperties(&p, cur));
  D->sms = p.multiProcessorCount;
  D->gpu_name = p.name;
  D->grid_small = D->sms * 8;
  SC_CUDA(cudaStreamCreateWithFlags(&D->capture, cudaStreamNonBlocking));

  const int nb = (int)L->boxes.size(), nd = (int)L->doms.size();
  std::vector<DBox> boxes(nb);
  D->box_wrap.assign(nb, 0);
  for (int b = 0; b < nb; ++b) {
    const sc_box& B = L->boxes[b];
    D->box_wrap[b] = (char)wrap_bits(L, b);
    boxes[b] = DBox{L->off[b], L->py[b], L->pz[b], (int)(B.hi[0] - B.lo[0]),
                    (int)(B.hi[1] - B.lo[1]), (int)(B.hi[2] - B.lo[2]), B.domain,
                    D->box_wrap[b]};
  }
  int rc = upload(&D->boxes, boxes);
  if (rc) return rc;

  auto index_of = [&](int b, const int64_t p[3]) {
    const sc_box& B = L->boxes[b];
    return L->off[b] + (p[0] - B.lo[0]) + (p[1] - B.lo[1]) * L->py[b] +
           (p[2] - B.lo[2]) * L->pz[b];
  };
  // ghost copies, chunked, grouped by destination box
  std::vector<DRect> grects;
  std::vector<DChunk> gchunks;
  std::vector<char> zface;  // per rect: it fills z ghosts of its box
  std::vector<char> xread;  // per rect: the warp-specialised kernels read it from its owner
  D->box_gchunks.assign(nb + 1, 0);
  {
    size_t c = 0;
    for (int b = 0; b < nb; ++b) {
      D->box_gchunks[b] = (int)gchunks.size();
      for (; c < L->copies.size() && L->copies[c].dst_box == b; ++c) {
        const sc_copy& C = L->copies[c];
        DRect r{};
        r.src = index_of(C.src_box, C.src_lo);
        r.dst = index_of(C.dst_box, C.dst_lo);
        r.spy = L->py[C.src_box];
        r.spz = L->pz[C.src_box];
        r.dpy = L->py[C.dst_box];
        r.dpz = L->pz[C.dst_box];
        r.ex = (int)C.ext[0];
        r.ey = (int)C.ext[1];
        r.ez = (int)C.ext[2];
        r.dom = L->boxes[b].domain;
        // 16-byte pairs when both ends of every row start on an even element
        // (pitches are multiples of 16 doubles)
        r.pairs = (C.ext[0] % 2 == 0 && r.src % 2 == 0 && r.dst % 2 == 0) ? 1 : 0;
        grects.push_back(r);
        zface.push_back(C.dst_lo[2] < L->boxes[b].lo[2] || C.dst_lo[2] >= L->boxes[b].hi[2]);
        xread.push_back(L->xread[c]);
        add_chunks((int)grects.size() - 1, (C.ext[0] >> r.pairs) * C.ext[1] * C.ext[2],
                   gchunks, dev::kGatherChunk);
      }
    }
    D->box_gchunks[nb] = (int)gchunks.size();
  }
  for (const DRect& r : grects)
    if (!rect_in_field(r.src, r.spy, r.spz, r.ex, r.ey, r.ez, L->field_size) ||
        !rect_in_field(r.dst, r.dpy, r.dpz, r.ex, r.ey, r.ez, L->field_size))
      return list_error("ghost-copy");
  rc = upload(&D->grects, grects);
  if (!rc) rc = upload(&D->gchunks, gchunks);
  if (rc) return rc;
  D->ngchunks = (int)gchunks.size();
  {
    // the exchange the stencil kernels need: every ghost of an ordinary
    // box, the z ghosts of a self-periodic one
    std::vector<DChunk> nw;
    for (int b = 0; b < nb; ++b)
      for (int c = D->box_gchunks[b]; c < D->box_gchunks[b + 1]; ++c)
        if (!D->box_wrap[b] || zface[gchunks[c].rect]) nw.push_back(gchunks[c]);
    D->ngchunks_nw = (int)nw.size();
    if (!nw.empty() && (rc = upload(&D->gchunks_nw, nw))) return rc;
    // the exchange the warp-specialised kernels need: every ghost of an
    // ordinary box, none of a self-periodic one (but the z ghosts of one of
    // a single plane)
    std::vector<DChunk> nzl;
    D->box_gchunks_nz.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
      D->box_gchunks_nz[b] = (int)nzl.size();
      for (int c = D->box_gchunks[b]; c < D->box_gchunks[b + 1]; ++c) {
        const int rr = gchunks[c].rect;
        if ((!D->box_wrap[b] && !xread[rr]) || (zface[rr] && !(D->box_wrap[b] & 2)))
          nzl.push_back(gchunks[c]);
      }
    }
    D->box_gchunks_nz[nb] = (int)nzl.size();
    D->ngchunks_nz = (int)nzl.size();
    if (!nzl.empty() && (rc = upload(&D->gchunks_nz, nzl))) return rc;
    // the x-face copies read from their owners, per box and side
    std::vector<DXGhost> xe;
    std::vector<int> xo(1, 0);
    for (int g = 0; g < 2 * nb; ++g) {
      xe.insert(xe.end(), L->xfaces[g].begin(), L->xfaces[g].end());
      xo.push_back((int)xe.size());
    }
    // the kernels read a source column over an item's planes and two more on
    // each side: the copy's source rows are interior rows of the source box,
    // so those planes lie in its padded block
    for (const DXGhost& e : xe)
      if (!rect_in_field((int64_t)e.src - 2 * (int64_t)e.spz, e.spy, e.spz, 2, e.y1 - e.y0,
                         e.z1 - e.z0 + 4, L->field_size))
        return list_error("x-face read");
    if (!xe.empty()) {
      if ((rc = upload(&D->xg, xe)) || (rc = upload(&D->xg_ofs, xo))) return rc;
    }
  }

  // the same copies seen from their sources: a ghost on the low (high) side
  // of its box along axis d is owned by a point in the high (low) two-deep
  // slab of the source box, so group the copies by (source box, d, slab)
  {
    std::vector<std::vector<DPush>> groups((size_t)nb * 6);
    for (const sc_copy& C : L->copies) {
      const sc_box& Bd = L->boxes[C.dst_box];
      const sc_box& Bs = L->boxes[C.src_box];
      int d = -1, side = 0;
      for (int a = 0; a < 3; ++a) {
        if (C.dst_lo[a] < Bd.lo[a]) { d = a; side = 1; }
        else if (C.dst_lo[a] >= Bd.hi[a]) { d = a; side = 0; }
      }
      if (d < 0) return set_error(SC_EINVAL, "exchange copy does not target a ghost region");
      // a self-periodic box's x and y ghosts are never read (the kernels
      // wrap those coordinates): push its z ghosts only
      if (D->box_wrap[C.dst_box] && d < 2) continue;
      DPush e{};
      e.lo0 = (int)(C.src_lo[0] - Bs.lo[0]);
      e.lo1 = (int)(C.src_lo[1] - Bs.lo[1]);
      e.lo2 = (int)(C.src_lo[2] - Bs.lo[2]);
      e.hi0 = e.lo0 + (int)C.ext[0];
      e.hi1 = e.lo1 + (int)C.ext[1];
      e.hi2 = e.lo2 + (int)C.ext[2];
      e.dbase = (int)index_of(C.dst_box, C.dst_lo);
      e.dpy = (int)L->py[C.dst_box];
      e.dpz = (int)L->pz[C.dst_box];
      // the kernels read sources inside the source box and write dbase onward
      if (e.lo0 < 0 || e.lo1 < 0 || e.lo2 < 0 || e.hi0 > Bs.hi[0] - Bs.lo[0] ||
          e.hi1 > Bs.hi[1] - Bs.lo[1] || e.hi2 > Bs.hi[2] - Bs.lo[2] ||
          !rect_in_field(e.dbase, e.dpy, e.dpz, C.ext[0], C.ext[1], C.ext[2], L->field_size))
        return list_error("ghost-push");
      groups[(size_t)C.src_box * 6 + 2 * d + side].push_back(e);
    }
    std::vector<DPush> entries;
    std::vector<int> gofs(1, 0);
    for (const auto& g : groups) {
      entries.insert(entries.end(), g.begin(), g.end());
      gofs.push_back((int)entries.size());
    }
    rc = upload(&D->push, entries);
    if (!rc) rc = upload(&D->push_gofs, gofs);
    if (rc) return rc;
  }

  // interior rectangles, and interior + six ghost slabs
  std::vector<DRect> irects, srects;
  std::vector<DChunk> ichunks, schunks, pchunks;
  for (int b = 0; b < nb; ++b) {
    const sc_box& B = L->boxes[b];
    int64_t n[3];
    for (int d = 0; d < 3; ++d) n[d] = B.hi[d] - B.lo[d];
    DRect r{};
    r.src = r.dst = L->off[b];
    r.spy = r.dpy = L->py[b];
    r.spz = r.dpz = L->pz[b];
    r.ex = (int)n[0];
    r.ey = (int)n[1];
    r.ez = (int)n[2];
    r.dom = B.domain;
    r.box = b;
    irects.push_back(r);
    add_chunks((int)irects.size() - 1, n[0] * n[1] * n[2], ichunks);
    add_chunks((int)irects.size() - 1, n[0] * n[1] * n[2], pchunks, dev::kGatherChunk);
    srects.push_back(r);
    add_chunks((int)srects.size() - 1, n[0] * n[1] * n[2], schunks);
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        int64_t p[3] = {B.lo[0], B.lo[1], B.lo[2]};
        p[d] = side ? B.hi[d] : B.lo[d] - 2;
        DRect s = r;
        s.src = s.dst = index_of(b, p);
        int e[3] = {(int)n[0], (int)n[1], (int)n[2]};
        e[d] = 2;
        s.ex = e[0];
        s.ey = e[1];
        s.ez = e[2];
        srects.push_back(s);
        add_chunks((int)srects.size() - 1, (int64_t)e[0] * e[1] * e[2], schunks);
      }
  }
  for (const DRect& r : irects)
    if (!rect_in_field(r.src, r.spy, r.spz, r.ex, r.ey, r.ez, L->field_size))
      return list_error("interior-rectangle");
  for (const DRect& r : srects)
    if (!rect_in_field(r.src, r.spy, r.spz, r.ex, r.ey, r.ez, L->field_size))
      return list_error("star-rectangle");
  rc = upload(&D->irects, irects);
  if (!rc) rc = upload(&D->ichunks, ichunks);
  if (!rc) rc = upload(&D->srects, srects);
  if (!rc) rc = upload(&D->schunks, schunks);
  if (!rc) rc = upload(&D->pchunks, pchunks);
  if (rc) return rc;
  D->npchunks = (int)pchunks.size();
  D->nichunks = (int)ichunks.size();
  D->nschunks = (int)schunks.size();

  if (L->partial && (rc = build_xfer_lists(L))) return rc;

  std::vector<double> inv(nd), h3(nd);
  for (int d = 0; d < nd; ++d) {
    const double h = L->doms[d].h;
    inv[d] = 1.0 / (12.0 * h * h);
    h3[d] = h * h * h;
  }
  rc = upload(&D->inv12h2, inv);
  if (!rc) rc = upload(&D->h3, h3);
  if (rc) return rc;
  SC_CUDA(cudaMalloc(&D->coef, sizeof(StageCoef) * 4 * nd));
  SC_CUDA(cudaMalloc(&D->qfac, sizeof(double) * 2 * nd));
  SC_CUDA(cudaMalloc(&D->emax, sizeof(unsigned) * 4 * nd));
  SC_CUDA(cudaMalloc(&D->emax_adj, sizeof(unsigned) * 8 * nd));
  SC_CUDA(cudaMalloc(&D->acoef, sizeof(dev::AdjCoef) * nd));
  SC_CUDA(cudaMemset(D->emax, 0, sizeof(unsigned) * 4 * nd));
  SC_CUDA(cudaMemset(D->emax_adj, 0, sizeof(unsigned) * 8 * nd));
  SC_CUDA(cudaMalloc(&D->err, sizeof(unsigned)));
  SC_CUDA(cudaMemset(D->err, 0, sizeof(unsigned)));
  SC_CUDA(cudaMalloc(&D->partial, sizeof(double) * std::max(1, D->nichunks)));
  D->pinned_size =
      sizeof(StageCoef) * 4 * nd + sizeof(double) * 2 * nd + sizeof(dev::AdjCoef) * nd + 64;
  SC_CUDA(cudaMallocHost(&D->pinned, D->pinned_size));
  return upload_items(L);
}

// Library-owned field buffer `name` (field_size doubles, zeroed once).
int get_field(sc_level* L, const std::string& name, double** p) {
  DeviceState* D = L->dev;
  auto it = D->fields.find(name);
  if (it != D->fields.end()) {
    *p = it->second;
    return SC_OK;
  }
  double* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(double) * L->field_size);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(SC_ENOMEM, "device allocation of scratch field '" + name + "' failed");
  }
  D->fields[name] = q;  // owned by the level from here, freed with it
  SC_CUDA(cudaMemset(q, 0, sizeof(double) * L->field_size));
  *p = q;
  return SC_OK;
}

// Per (stage, domain) coefficients for step sizes dt (ndt == 1 or ndom).
int set_coef(sc_level* L, const double* dt, int ndt, cudaStream_t s) {
  DeviceState* D = L->dev;
  const int nd = (int)L->doms.size();
  if (!dt || (ndt != 1 && ndt != nd)) return set_error(SC_EINVAL, "dt must have 1 or ndom entries");
  std::vector<double> want(nd);
  for (int d = 0; d < nd; ++d) {
    want[d] = dt[ndt == 1 ? 0 : d];
    if (!(want[d] > 0.0) && want[d] != 0.0) return set_error(SC_EINVAL, "dt must be >= 0");
  }
  if (want == D->coef_dt) return SC_OK;
  static const double c[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
  static const int qk[4] = {-2, 0, -1, 0};  // stage factors folded into the stencil sum
  // wait for earlier work that reads the pinned staging buffer
  SC_CUDA(cudaStreamSynchronize(s));
  StageCoef* h = reinterpret_cast<StageCoef*>(D->pinned);
  double* qf = reinterpret_cast<double*>(h + 4 * nd);
  dev::AdjCoef* ac = reinterpret_cast<dev::AdjCoef*>(qf + 2 * nd);
  for (int d = 0; d < nd; ++d) {
    const double hh = L->doms[d].h;
    const double inv = 1.0 / (12.0 * hh * hh);
    double g[4];
    for (int st = 0; st < 4; ++st) g[st] = c[st] * want[d];
    // adjoint constants: G4, G34, G234, G1234 (products of the stage steps)
    const double G4 = g[3], G34 = g[2] * g[3], G234 = g[1] * G34, G1234 = g[0] * G234;
    const double C[4] = {G1234 * inv, G234 * inv, G34, G4};  // of Lw0 .. Lw3
    for (int st = 0; st < 4; ++st)
      h[st * nd + d] = StageCoef{g[st], g[st] * inv, inv, C[st] * std::ldexp(1.0, -qk[st]) * inv};
    qf[2 * d] = want[d] * inv;
    qf[2 * d + 1] = (want[d] / 3.0) * inv;
    ac[d] = dev::AdjCoef{{G4 * inv, G34 * inv, G234 * inv * inv, G1234 * inv * inv},
                         {G4, G34 * inv, G234 * inv, G1234 * inv * inv}};
  }
  SC_CUDA(cudaMemcpyAsync(D->coef, h, sizeof(StageCoef) * 4 * nd, cudaMemcpyHostToDevice, s));
  SC_CUDA(cudaMemcpyAsync(D->qfac, qf, sizeof(double) * 2 * nd, cudaMemcpyHostToDevice, s));
  SC_CUDA(cudaMemcpyAsync(D->acoef, ac, sizeof(dev::AdjCoef) * nd, cudaMemcpyHostToDevice, s));
  D->coef_dt = want;
  return SC_OK;
}

static bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// ---- enqueueing ------------------------------------------------------------

struct Enq {
  sc_level* L;
  cudaStream_t s;
  int64_t* count;
  bool per_box;
  bool timed = false;
  // ghost exchange of the stage outputs: false = a gather launch before each
  // stage (best when a CUDA graph hides the launches), true = every stage
  // kernel writes the ghost copies of what it produces (fewer launches)
  bool push = false;
  // recompute the pre-scaled wave speeds in the prologue (false: a caller
  // that keeps c2 and dt knows they are current)
  bool qprep = true;
  // gathers refresh the ghosts of every box (sc_level_fill_ghosts); false:
  // only those the stencil kernels read (not those of self-periodic boxes)
  bool all_ghosts = false;
  // the exponent bounds of the run's input are already in place (see
  // level_steps)
  bool bounds = false;
};

// Event pair around one launch when timing is on.
struct TimedLaunch {
  const Enq& q;
  cudaEvent_t e1 = nullptr;
  TimedLaunch(const Enq& q_, int kind) : q(q_) {
    if (!q.timed) return;
    DeviceState* D = q.L->dev;
    if (D->ev_used == D->ev_pool.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      D->ev_pool.emplace_back(a, b);
    }
    auto& pr = D->ev_pool[D->ev_used++];
    D->ev_kind.push_back(kind);
    cudaEventRecord(pr.first, q.s);
    e1 = pr.second;
  }
  ~TimedLaunch() {
    if (e1) cudaEventRecord(e1, q.s);
  }
};

static cudaError_t enq_fill(const Enq& q, double* f) {
  DeviceState* D = q.L->dev;
  if (!q.per_box) {
    const int n = q.all_ghosts ? D->ngchunks : D->ngchunks_nw;
    if (n <= 0) return cudaSuccess;
    (*q.count)++;
    TimedLaunch t(q, SC_KERNEL_GATHER);
    return dev::launch_gather(D->grects, q.all_ghosts ? D->gchunks : D->gchunks_nw, n, f,
                              D->grid_small, q.s);
  }
  for (size_t b = 0; b + 1 < D->box_gchunks.size(); ++b) {
    const int n = D->box_gchunks[b + 1] - D->box_gchunks[b];
    if (n <= 0) continue;  // per box: every ghost (simplest; not the fast path)
    (*q.count)++;
    TimedLaunch t(q, SC_KERNEL_GATHER);
    cudaError_t e = dev::launch_gather(D->grects, D->gchunks + D->box_gchunks[b], n, f,
                                       D->grid_small, q.s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t enq_maxexp(const Enq& q, const double* f, unsigned* slot, bool star) {
  DeviceState* D = q.L->dev;
  (*q.count)++;
  if (star)
    return dev::launch_maxexp(D->srects, D->schunks, D->nschunks, f, slot, D->err,
                              D->grid_small, q.s);
  return dev::launch_maxexp(D->irects, D->ichunks, D->nichunks, f, slot, D->err, D->grid_small,
                            q.s);
}

static cudaError_t enq_fwd(const Enq& q, dev::FwdArgs a, bool record) {
  DeviceState* D = q.L->dev;
  if (!q.per_box) {
    a.items = D->items;
    a.nitems = D->nitems;
    (*q.count)++;
    TimedLaunch t(q, record ? SC_KERNEL_STAGE_RECORD : SC_KERNEL_STAGE);
    return dev::launch_fwd_stage(q.L->arith, record, q.L->staging, a,
                                 D->grid_stage_s[q.L->staging], q.s);
  }
  for (size_t b = 0; b + 1 < D->box_items.size(); ++b) {
    a.items = D->items_box + D->box_items[b];
    a.nitems = D->box_items[b + 1] - D->box_items[b];
    (*q.count)++;
    TimedLaunch t(q, record ? SC_KERNEL_STAGE_RECORD : SC_KERNEL_STAGE);
    cudaError_t e = dev::launch_fwd_stage(q.L->arith, record, q.L->staging, a,
                                          D->grid_stage_s[q.L->staging], q.s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One RK4 step in nested form on (u, pi), stage scratch Wa, Wb.  If lapw is
// not NULL, stage s also records L w_{s-1}.u into lapw[s].
static cudaError_t enq_step(const Enq& q, double* u, double* pi, const double* c2,
                            double* const* W, double* const* lapw) {
  DeviceState* D = q.L->dev;
  const int nd = (int)q.L->doms.size();
  // stage factors c_s = 1/4, 1/3, 1/2, 1: powers of two fold into the
  // exponent of the Laplacian; 1/3 is in the second pre-scaled array
  const double* qarr[4] = {W[4], W[5], W[4], W[4]};
  const int qk[4] = {-2, 0, -1, 0};
  double* in_u[4] = {u, W[0], W[2], W[0]};
  double* in_p[4] = {pi, W[1], W[3], W[1]};
  double* out_u[4] = {W[0], W[2], W[0], u};
  double* out_p[4] = {W[1], W[3], W[1], pi};
  // with push, each stage writes the ghosts of its stencil output, so the
  // next stage (and the next step) find theirs filled and only the first
  // input of a run is gathered (enq_prologue); otherwise each stage gathers
  for (int s = 0; s < 4; ++s) {
    cudaError_t e;
    if (!q.push) {
      e = enq_fill(q, in_u[s]);
      if (e != cudaSuccess) return e;
    }
    dev::FwdArgs a{};
    a.ndom = nd;
    a.boxes = D->boxes;
    a.wu_in = in_u[s];
    a.wp_in = in_p[s];
    a.yu = u;
    a.yp = pi;
    a.c2 = c2;
    a.wu_out = out_u[s];
    a.wp_out = out_p[s];
    a.lapw = lapw ? lapw[s] : nullptr;
    a.q = qarr[s];
    a.qk = qk[s];
    a.push = q.push ? D->push : nullptr;
    a.push_gofs = q.push ? D->push_gofs : nullptr;
    a.coef = D->coef + s * nd;
    a.emax_in = D->emax + (s % 4) * nd;
    a.emax_out = D->emax + ((s + 1) % 4) * nd;
    a.emax_clear = D->emax + ((s + 2) % 4) * nd;
    a.err = D->err;
    e = enq_fwd(q, a, lapw != nullptr);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Ghost gather of two fields; the exponent slots `clear` (2 ndom, may be
// NULL) are zeroed for the kernel that follows.
static cudaError_t enq_fill2(const Enq& q, double* f, double* g, unsigned* clear) {
  DeviceState* D = q.L->dev;
  const int nclear = clear ? 2 * (int)q.L->doms.size() : 0;
  bool cleared = clear == nullptr;
  if (!q.per_box) {
    // the pass kernels that follow read what is gathered here
    const bool ws = q.L->pass_ws && !q.all_ghosts;
    const int n = q.all_ghosts ? D->ngchunks : (ws ? D->ngchunks_nz : D->ngchunks_nw);
    const DChunk* list = q.all_ghosts ? D->gchunks : (ws ? D->gchunks_nz : D->gchunks_nw);
    if (n > 0) {
      (*q.count)++;
      TimedLaunch t(q, SC_KERNEL_GATHER);
      cudaError_t e = dev::launch_gather2(D->grects, list, n, f, g, clear, nclear, q.s);
      if (e != cudaSuccess) return e;
      cleared = true;
    }
  } else {
    // one launch per box: the box's part of the same list (every ghost of
    // the box where the one-role kernels follow or every ghost is wanted)
    const bool ws = q.L->pass_ws && !q.all_ghosts;
    const std::vector<int>& off = ws ? D->box_gchunks_nz : D->box_gchunks;
    const DChunk* list = ws ? D->gchunks_nz : D->gchunks;
    for (size_t b = 0; b + 1 < off.size(); ++b) {
      const int n = off[b + 1] - off[b];
      if (n <= 0) continue;
      (*q.count)++;
      TimedLaunch t(q, SC_KERNEL_GATHER);
      cudaError_t e = dev::launch_gather2(D->grects, list + off[b], n, f, g,
                                          cleared ? nullptr : clear, nclear, q.s);
      if (e != cudaSuccess) return e;
      cleared = true;
    }
  }
  if (!cleared) return cudaMemsetAsync(clear, 0, sizeof(unsigned) * nclear, q.s);
  return cudaSuccess;
}

static cudaError_t enq_pair(const Enq& q, dev::PairArgs a, bool second) {
  DeviceState* D = q.L->dev;
  const int kind = second ? SC_KERNEL_PAIR_B : SC_KERNEL_PAIR_A;
  if (!q.per_box) {
    a.items = D->items;
    a.nitems = D->nitems;
    (*q.count)++;
    TimedLaunch t(q, kind);
    return launch_pass(q.L, second, a, q.s);
  }
  for (size_t b = 0; b + 1 < D->box_items.size(); ++b) {
    a.items = D->items_box + D->box_items[b];
    a.nitems = D->box_items[b + 1] - D->box_items[b];
    (*q.count)++;
    TimedLaunch t(q, kind);
    cudaError_t e = launch_pass(q.L, second, a, q.s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One RK4 step in two passes of two stages each (see kernels.cu): W[0], W[1]
// receive w_2, W[2] receives 12 h^2 L y.u.  Exponent slots: X = emax[0, 2
// ndom) holds the bounds of (u, pi), Y = emax[2 ndom, 4 ndom) those of w_2;
// each gather zeroes the slots that the pass after it accumulates into.  If
// lapw is not NULL, lapw[s] receives C_{s+1} L w_s.u as enq_step records it.
static cudaError_t enq_pass(const Enq& q, double* u, double* pi, double* const* W, int pass,
                            double* const* lapw = nullptr) {
  DeviceState* D = q.L->dev;
  const int nd = (int)q.L->doms.size();
  const bool fixed = q.L->arith == SC_ARITH_FIXED;
  unsigned* X = D->emax;
  unsigned* Y = D->emax + 2 * nd;
  dev::PairArgs a{};
  a.ndom = nd;
  a.boxes = D->boxes;
  a.yu = u;
  a.yp = pi;
  a.q = W[4];
  a.coef = D->coef;
  a.err = D->err;
  a.xg = D->xg;
  a.xg_ofs = D->xg_ofs;
  if (pass == 0) {
    cudaError_t e = enq_fill2(q, u, pi, fixed ? Y : nullptr);
    if (e != cudaSuccess) return e;
    a.s0 = u;
    a.s1 = pi;
    a.x = W[5];
    a.out_u = W[0];
    a.out_p = W[1];
    a.ly = W[2];
    a.emax_in = X;
    a.emax_out = Y;
    a.rec0 = lapw ? lapw[0] : nullptr;
    a.rec1 = lapw ? lapw[1] : nullptr;
    return enq_pair(q, a, false);
  }
  cudaError_t e = enq_fill2(q, W[0], W[1], fixed ? X : nullptr);
  if (e != cudaSuccess) return e;
  a.s0 = W[0];
  a.s1 = W[1];
  a.x = W[2];
  a.out_u = u;
  a.out_p = pi;
  a.ly = nullptr;
  a.emax_in = Y;
  a.emax_out = X;
  a.rec0 = lapw ? lapw[2] : nullptr;
  a.rec1 = lapw ? lapw[3] : nullptr;
  return enq_pair(q, a, true);
}

static cudaError_t enq_step_pairs(const Enq& q, double* u, double* pi, double* const* W,
                                  double* const* lapw = nullptr) {
  cudaError_t e = enq_pass(q, u, pi, W, 0, lapw);
  if (e != cudaSuccess) return e;
  return enq_pass(q, u, pi, W, 1, lapw);
}

// Prologue of a run of steps: the ghosts of u gathered (push exchange); the
// pre-scaled wave speed q = c2 * dt/(12 h^2) (and the 1/3 variant) in W[4],
// W[5]; for the fixed form, the exponent ring cleared and slot 0 = max
// exponent of u (and, if pi is not NULL, slot ndom = that of pi).
static cudaError_t enq_prologue(const Enq& q, double* u, double* pi, const double* c2,
                                double* const* W) {
  DeviceState* D = q.L->dev;
  if (q.push) {
    cudaError_t e0 = enq_fill(q, u);  // ghosts of the run's first stencil input
    if (e0 != cudaSuccess) return e0;
  }
  cudaError_t e = cudaSuccess;
  if (q.qprep) {
    (*q.count)++;
    e = dev::launch_qprep(D->irects, D->ichunks, D->nichunks, c2, W[4], W[5], D->qfac,
                          D->grid_small, q.s);
    if (e != cudaSuccess) return e;
  }
  if (q.L->arith != SC_ARITH_FIXED) return cudaSuccess;
  if (q.bounds && pi && q.L->fuse == 2) return cudaSuccess;  // slots X hold them
  e = cudaMemsetAsync(D->emax, 0, sizeof(unsigned) * 4 * q.L->doms.size(), q.s);
  if (e != cudaSuccess) return e;
  // With a non-periodic domain the boundary ghosts hold caller data that
  // the stencils read: the bound then covers interior and ghosts, taken
  // after an exchange has refreshed the owned ghosts.
  const bool star = !q.L->all_periodic;
  if (star && !q.push) {
    e = pi ? enq_fill2(q, u, pi, nullptr) : enq_fill(q, u);
    if (e != cudaSuccess) return e;
  }
  e = enq_maxexp(q, u, D->emax, star);
  if (e != cudaSuccess || !pi) return e;
  return enq_maxexp(q, pi, D->emax + q.L->doms.size(), star);  // slot X.pi of the pair form
}

// Stage scratch: Wa.u, Wa.pi, Wb.u, Wb.pi and the two pre-scaled wave speeds.
int scratch4(sc_level* L, double* W[6]) {
  const char* names[6] = {"Wa.u", "Wa.pi", "Wb.u", "Wb.pi", "q.a", "q.b"};
  for (int i = 0; i < 6; ++i) {
    int rc = get_field(L, names[i], &W[i]);
    if (rc) return rc;
  }
  return SC_OK;
}

static int run_steps(sc_level* L, double* u, double* pi, const double* c2, int nsteps, int mode,
                     cudaStream_t s, bool qprep = true, bool bounds = false) {
  DeviceState* D = L->dev;
  double* W[6];
  int rc = scratch4(L, W);
  if (rc) return rc;
  Enq q{L, s, &L->launches, mode == SC_MODE_PER_BOX};
  q.qprep = qprep;
  q.bounds = bounds;
  if (mode == SC_MODE_TIMED) {
    q.timed = true;
    D->ev_used = 0;
    D->ev_kind.clear();
  }
  const bool pairs = L->fuse == 2;
  SC_CUDA(enq_prologue(q, u, pairs ? pi : nullptr, c2, W));
  auto step = [&](const Enq& e) {
    return pairs ? enq_step_pairs(e, u, pi, W) : enq_step(e, u, pi, c2, W, nullptr);
  };
  if (mode != SC_MODE_GRAPH) {
    for (int n = 0; n < nsteps; ++n) SC_CUDA(step(q));
    return SC_OK;
  }
  auto key = std::make_tuple((const void*)u, (const void*)pi, (const void*)c2,
                             L->arith + 2 * L->fuse + 4 * L->staging + 8 * L->pass_ws,
                             L->version);
  auto it = D->graphs.find(key);
  if (it == D->graphs.end()) {
    if (D->graphs.size() >= 16) {  // bounded cache: start it afresh
      SC_CUDA(cudaStreamSynchronize(s));
      for (auto& kv : D->graphs) cudaGraphExecDestroy(kv.second.first);
      D->graphs.clear();
    }
    int64_t nodes = 0;
    Enq cq{L, D->capture, &nodes, false};
    SC_CUDA(cudaStreamBeginCapture(D->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = step(cq);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(D->capture, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "capture of the RK4 step");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    it = D->graphs.emplace(key, std::make_pair(ex, (int)nodes)).first;
  }
  for (int n = 0; n < nsteps; ++n) {
    SC_CUDA(cudaGraphLaunch(it->second.first, s));
    L->launches += it->second.second;
  }
  return SC_OK;
}

int level_steps(sc_level* L, double* u, double* pi, const double* c2, double dt, int nsteps,
                int mode, cudaStream_t s, bool qprep, bool bounds) {
  int rc = sc_level_rk4_step(L, u, pi, c2, &dt, 1, 0, mode, s);  // validation and set-up
  if (rc || nsteps == 0) return rc;
  return run_steps(L, u, pi, c2, nsteps, mode, s, qprep, bounds);
}

}  // namespace sc

using namespace sc;

extern "C" {

int sc_level_work_items(const sc_level* L, int32_t* out, int64_t cap, int64_t* n) {
  if (!L || !n) return set_error(SC_EINVAL, "NULL argument");
  if (cap > 0 && !out) return set_error(SC_EINVAL, "out is NULL");
  std::vector<DItem> items;
  std::vector<int> box_items;
  build_items(L, items, box_items);
  order_items(L, items);
  *n = (int64_t)items.size();
  const int64_t m = std::min<int64_t>(cap, *n);
  for (int64_t i = 0; i < m; ++i) {
    const DItem& it = items[(size_t)i];
    const int32_t row[6] = {it.box, it.x0, it.y0, it.z0, it.nzr, 2 * it.txh};
    std::memcpy(out + 6 * i, row, sizeof(row));
  }
  return SC_OK;
}

int sc_level_fill_ghosts(sc_level* L, double* field, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!aligned16(field)) return set_error(SC_EINVAL, "field must be a 16-byte aligned pointer");
  int rc = ensure_device(L);
  if (rc) return rc;
  Enq q{L, (cudaStream_t)stream, &L->launches, false};
  q.all_ghosts = true;
  SC_CUDA(enq_fill(q, field));
  return SC_OK;
}

int sc_level_apply_laplacian(sc_level* L, const double* u, double* out, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!aligned16(u) || !aligned16(out))
    return set_error(SC_EINVAL, "fields must be 16-byte aligned pointers");
  if (u == out) return set_error(SC_EINVAL, "u and out must not overlap");
  int rc = ensure_device(L);
  if (rc) return rc;
  DeviceState* D = L->dev;
  cudaStream_t s = (cudaStream_t)stream;
  Enq q{L, s, &L->launches, false};
  const int nd = (int)L->doms.size();
  if (L->arith == SC_ARITH_FIXED) {
    SC_CUDA(cudaMemsetAsync(D->emax, 0, sizeof(unsigned) * 4 * nd, s));
    SC_CUDA(enq_maxexp(q, u, D->emax, true));
  }
  dev::LapArgs a{D->items, D->nitems, nd, D->boxes, u, out, D->inv12h2, D->emax, D->err};
  L->launches++;
  SC_CUDA(dev::launch_lap(L->arith, a, D->grid_stage, s));
  return SC_OK;
}

int sc_level_rk4_step(sc_level* L, double* u, double* pi, const double* c2, const double* dt,
                      int32_t ndt, int32_t nsteps, int32_t mode, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!aligned16(u) || !aligned16(pi) || !aligned16(c2))
    return set_error(SC_EINVAL, "u, pi, c2 must be 16-byte aligned device pointers");
  if (nsteps < 0) return set_error(SC_EINVAL, "nsteps < 0");
  if (mode != SC_MODE_GRAPH && mode != SC_MODE_PER_BOX && mode != SC_MODE_BATCHED &&
      mode != SC_MODE_TIMED)
    return set_error(SC_EINVAL, "unknown mode");
  if (!L->all_periodic && nsteps > 1)
    return set_error(SC_EINVAL,
                     "a level with a non-periodic domain takes one step per call (its "
                     "boundary ghosts are refreshed between steps)");
  if (L->partial)
    return set_error(SC_EINVAL,
                     "distributed level: step it with sc_dist_rk4_begin and sc_dist_rk4_pass, "
                     "with the exchange of sc_dist_pack / sc_dist_unpack between passes");
  int rc = ensure_device(L);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = set_coef(L, dt, ndt, s);
  if (rc) return rc;
  if (nsteps == 0) return SC_OK;
  return run_steps(L, u, pi, c2, nsteps, mode, s);
}

int sc_level_rk4_step_host(sc_level* L, const double* u, const double* pi, const double* c2,
                           double* u_out, double* pi_out, const double* dt, int32_t ndt,
                           int32_t nsteps, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!u || !pi || !c2 || !u_out || !pi_out) return set_error(SC_EINVAL, "NULL host buffer");
  int rc = ensure_device(L);
  if (rc) return rc;
  double *du, *dp, *dc;
  if ((rc = get_field(L, "host.u", &du)) || (rc = get_field(L, "host.pi", &dp)) ||
      (rc = get_field(L, "host.c2", &dc)))
    return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * L->field_size;
  SC_CUDA(cudaMemcpyAsync(du, u, bytes, cudaMemcpyHostToDevice, s));
  SC_CUDA(cudaMemcpyAsync(dp, pi, bytes, cudaMemcpyHostToDevice, s));
  SC_CUDA(cudaMemcpyAsync(dc, c2, bytes, cudaMemcpyHostToDevice, s));
  rc = sc_level_rk4_step(L, du, dp, dc, dt, ndt, nsteps, SC_MODE_GRAPH, stream);
  if (rc) return rc;
  SC_CUDA(cudaMemcpyAsync(u_out, du, bytes, cudaMemcpyDeviceToHost, s));
  SC_CUDA(cudaMemcpyAsync(pi_out, dp, bytes, cudaMemcpyDeviceToHost, s));
  return sc_level_sync(L, stream);
}

int sc_level_misfit(sc_level* L, const double* u, const double* u_obs, double* loss,
                    double* seed, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!aligned16(u) || !aligned16(u_obs) || !loss || (seed && !aligned16(seed)))
    return set_error(SC_EINVAL, "bad pointer");
  int rc = ensure_device(L);
  if (rc) return rc;
  DeviceState* D = L->dev;
  L->launches += 2;
  SC_CUDA(dev::launch_misfit(D->irects, D->ichunks, D->nichunks, u, u_obs, seed, D->h3,
                             D->partial, loss, D->grid_small, (cudaStream_t)stream));
  return SC_OK;
}

int sc_level_sync(sc_level* L, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!L->dev) return SC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* h = reinterpret_cast<unsigned*>(L->dev->pinned) +
                (L->dev->pinned_size / sizeof(unsigned) - 4);
  SC_CUDA(cudaMemcpyAsync(h, L->dev->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  SC_CUDA(cudaStreamSynchronize(s));
  const unsigned e = *h;
  if (e) {
    SC_CUDA(cudaMemset(L->dev->err, 0, sizeof(unsigned)));
    std::string m = "device error word set:";
    if (e & dev::kErrNonFinite) m += " non-finite value in the fixed-point Laplacian;";
    if (e & dev::kErrScale) m += " input above its domain's exponent bound;";
    if (e & dev::kErrBounds) m += " index outside its box (checked build);";
    if (e & dev::kErrTimeout) m += " a bounded wait inside a kernel gave up;";
    return set_error(SC_EDEVICE, m);
  }
  return SC_OK;
}

// ---- distributed level: exchange and split step ------------------------

static int dist_fields(sc_level* L, int32_t which, const double* u, const double* pi,
                       double** f, double** g) {
  if (which == SC_DIST_STATE) {
    if (!aligned16(u) || !aligned16(pi))
      return set_error(SC_EINVAL, "u, pi must be 16-byte aligned device pointers");
    *f = const_cast<double*>(u);
    *g = const_cast<double*>(pi);
    return SC_OK;
  }
  if (which != SC_DIST_STAGE) return set_error(SC_EINVAL, "which must be SC_DIST_STATE or SC_DIST_STAGE");
  double* W[6];
  const int rc = scratch4(L, W);
  if (rc) return rc;
  *f = W[0];
  *g = W[1];
  return SC_OK;
}

static int dist_xfer(sc_level* L, bool pack, int32_t which, const double* u, const double* pi,
                     double* buf, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!L->partial) return set_error(SC_EINVAL, "not a distributed level (sc_dist_create)");
  const int64_t need = pack ? L->send_doubles : L->recv_doubles;
  if (need > 0 && (!buf || (reinterpret_cast<uintptr_t>(buf) & 7)))
    return set_error(SC_EINVAL, "exchange buffer must be an 8-byte aligned device pointer");
  int rc = ensure_device(L);
  if (rc) return rc;
  double *f, *g;
  if ((rc = dist_fields(L, which, u, pi, &f, &g))) return rc;
  DeviceState* D = L->dev;
  const int nd = (int)L->doms.size();
  unsigned* emax = nullptr;
  if (!pack && L->arith == SC_ARITH_FIXED)  // X: bounds of (u, pi); Y: of w_2
    emax = which == SC_DIST_STATE ? D->emax : D->emax + 2 * nd;
  const int n = pack ? D->nxsend_chunks : D->nxrecv_chunks;
  if (n > 0) L->launches++;
  SC_CUDA(dev::launch_xfer(pack, pack ? D->xsend : D->xrecv,
                           pack ? D->xsend_chunks : D->xrecv_chunks, n, f, g, buf, emax, nd,
                           D->grid_small, (cudaStream_t)stream));
  return SC_OK;
}

int sc_dist_pack(sc_level* L, int32_t which, const double* u, const double* pi, double* send,
                 void* stream) {
  return dist_xfer(L, true, which, u, pi, send, stream);
}

int sc_dist_unpack(sc_level* L, int32_t which, const double* recv, double* u, double* pi,
                   void* stream) {
  return dist_xfer(L, false, which, u, pi, const_cast<double*>(recv), stream);
}

int sc_dist_rk4_begin(sc_level* L, double* u, double* pi, const double* c2, const double* dt,
                      int32_t ndt, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!L->partial) return set_error(SC_EINVAL, "not a distributed level (sc_dist_create)");
  if (!aligned16(u) || !aligned16(pi) || !aligned16(c2))
    return set_error(SC_EINVAL, "u, pi, c2 must be 16-byte aligned device pointers");
  if (u == pi) return set_error(SC_EINVAL, "u and pi must be different buffers");
  L->dist_begun = false;
  int rc = ensure_device(L);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = set_coef(L, dt, ndt, s))) return rc;
  double* W[6];
  if ((rc = scratch4(L, W))) return rc;
  Enq q{L, s, &L->launches, false};
  SC_CUDA(enq_prologue(q, u, pi, c2, W));
  L->dist_begun = true;
  L->dist_next_pass = 0;
  L->dist_u = u;
  L->dist_pi = pi;
  return SC_OK;
}

int sc_dist_rk4_pass(sc_level* L, double* u, double* pi, int32_t pass, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!L->partial) return set_error(SC_EINVAL, "not a distributed level (sc_dist_create)");
  if (!L->dist_begun) return set_error(SC_EINVAL, "no run: call sc_dist_rk4_begin first");
  if (pass != 0 && pass != 1) return set_error(SC_EINVAL, "pass must be 0 or 1");
  if (pass != L->dist_next_pass)
    return set_error(SC_EINVAL, pass ? "pass 1 needs pass 0 of the step first"
                                     : "pass 0 needs the previous step's pass 1 first");
  if (u != L->dist_u || pi != L->dist_pi)
    return set_error(SC_EINVAL, "u, pi must be the buffers given to sc_dist_rk4_begin");
  double* W[6];
  int rc = scratch4(L, W);
  if (rc) return rc;
  Enq q{L, (cudaStream_t)stream, &L->launches, false};
  SC_CUDA(enq_pass(q, u, pi, W, pass));
  L->dist_next_pass = 1 - pass;
  return SC_OK;
}

// Forward sweep keeping a checkpoint every K steps (the tape of the level).
int sc_level_forward_tape(sc_level* L, const double* u0, const double* pi0, const double* c2,
                          const double* dt, int32_t ndt, int32_t nsteps, int32_t ckpt_every,
                          double* u_T, double* pi_T, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!aligned16(u0) || !aligned16(pi0) || !aligned16(c2) || (u_T && !aligned16(u_T)) ||
      (pi_T && !aligned16(pi_T)))
    return set_error(SC_EINVAL, "fields must be 16-byte aligned device pointers");
  if (nsteps < 0 || ckpt_every < 1) return set_error(SC_EINVAL, "nsteps < 0 or ckpt_every < 1");
  if (!L->all_periodic) return set_error(SC_EINVAL, "needs domains periodic on every axis");
  if (L->partial) return set_error(SC_EINVAL, "the adjoint of a distributed level is not built");
  int rc = ensure_device(L);
  if (rc) return rc;
  DeviceState* D = L->dev;
  cudaStream_t s = (cudaStream_t)stream;
  rc = set_coef(L, dt, ndt, s);
  if (rc) return rc;
  const int K = ckpt_every;
  const int nck = (nsteps + K - 1) / K;
  const size_t bytes = sizeof(double) * L->field_size;
  double *W[6], *Su, *Sp;
  if ((rc = scratch4(L, W)) || (rc = get_field(L, "S.u", &Su)) ||
      (rc = get_field(L, "S.pi", &Sp)))
    return rc;
  std::vector<double*> cku(nck), ckp(nck);
  for (int c = 0; c < nck; ++c)
    if ((rc = get_field(L, "ck.u." + std::to_string(c), &cku[c])) ||
        (rc = get_field(L, "ck.pi." + std::to_string(c), &ckp[c])))
      return rc;
  L->tape_valid = false;
  // two stages per pass exchange ghosts by gathers; one stage per pass has
  // each stage kernel push the ghosts of what it writes
  const bool pairs = L->fuse == 2;
  Enq q{L, s, &L->launches, false};
  q.push = !pairs;
  if (L->profile) {
    q.timed = true;
    D->ev_used = 0;
    D->ev_kind.clear();
  }
  SC_CUDA(cudaMemcpyAsync(Su, u0, bytes, cudaMemcpyDeviceToDevice, s));
  SC_CUDA(cudaMemcpyAsync(Sp, pi0, bytes, cudaMemcpyDeviceToDevice, s));
  for (int c = 0; c < nck; ++c) {
    const int len = std::min(K, nsteps - c * K);
    SC_CUDA(cudaMemcpyAsync(cku[c], Su, bytes, cudaMemcpyDeviceToDevice, s));
    SC_CUDA(cudaMemcpyAsync(ckp[c], Sp, bytes, cudaMemcpyDeviceToDevice, s));
    SC_CUDA(enq_prologue(q, Su, pairs ? Sp : nullptr, c2, W));
    for (int n = 0; n < len; ++n)
      SC_CUDA(pairs ? enq_step_pairs(q, Su, Sp, W) : enq_step(q, Su, Sp, c2, W, nullptr));
  }
  if (u_T) SC_CUDA(cudaMemcpyAsync(u_T, Su, bytes, cudaMemcpyDeviceToDevice, s));
  if (pi_T) SC_CUDA(cudaMemcpyAsync(pi_T, Sp, bytes, cudaMemcpyDeviceToDevice, s));
  L->tape_valid = true;
  L->tape_nsteps = nsteps;
  L->tape_ckpt = K;
  L->tape_c2 = c2;
  L->tape_dt = D->coef_dt;
  return SC_OK;
}

// Reverse sweep over the tape of the last sc_level_forward_tape.
int sc_level_backward_tape(sc_level* L, const double* c2, const double* gu_T,
                           const double* gpi_T, double* g_u0, double* g_pi0, double* g_c2,
                           void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!L->tape_valid) return set_error(SC_EINVAL, "no forward tape: call sc_level_forward_tape");
  if (c2 != L->tape_c2) return set_error(SC_EINVAL, "c2 differs from the taped forward's");
  if (!aligned16(g_u0) || !aligned16(g_pi0) || !aligned16(g_c2) || (gu_T && !aligned16(gu_T)) ||
      (gpi_T && !aligned16(gpi_T)))
    return set_error(SC_EINVAL, "fields must be 16-byte aligned device pointers");
  int rc = ensure_device(L);
  if (rc) return rc;
  DeviceState* D = L->dev;
  cudaStream_t s = (cudaStream_t)stream;
  const int nd = (int)L->doms.size();
  rc = set_coef(L, L->tape_dt.data(), nd, s);
  if (rc) return rc;
  const int nsteps = L->tape_nsteps, K = L->tape_ckpt;
  const int nck = (nsteps + K - 1) / K;
  const size_t bytes = sizeof(double) * L->field_size;
  double *W[6], *Su, *Sp, *Yu, *Yp, *Za, *Zb, *L1, *L2, *L3;
  if ((rc = scratch4(L, W)) || (rc = get_field(L, "S.u", &Su)) ||
      (rc = get_field(L, "S.pi", &Sp)) || (rc = get_field(L, "Y.u", &Yu)) ||
      (rc = get_field(L, "Y.pi", &Yp)) || (rc = get_field(L, "Za", &Za)) ||
      (rc = get_field(L, "Zb", &Zb)) || (rc = get_field(L, "L1", &L1)) ||
      (rc = get_field(L, "L2", &L2)) || (rc = get_field(L, "L3", &L3)))
    return rc;
  std::vector<double*> cku(nck), ckp(nck), lapw(4 * std::min(K, std::max(nsteps, 1)));
  for (int c = 0; c < nck; ++c)
    if ((rc = get_field(L, "ck.u." + std::to_string(c), &cku[c])) ||
        (rc = get_field(L, "ck.pi." + std::to_string(c), &ckp[c])))
      return rc;
  for (size_t j = 0; j < lapw.size(); ++j)
    if ((rc = get_field(L, "lapw." + std::to_string(j), &lapw[j]))) return rc;

  Enq q{L, s, &L->launches, false};
  q.push = true;
  if (L->profile) {
    q.timed = true;
    D->ev_used = 0;
    D->ev_kind.clear();
  }
  const bool fixed = L->arith == SC_ARITH_FIXED;
  const bool pairs = L->fuse == 2;  // form of the forward recomputation
  double *P4, *P3, *P2, *P1;
  if ((rc = get_field(L, "P4", &P4)) || (rc = get_field(L, "P3", &P3)) ||
      (rc = get_field(L, "P2", &P2)) || (rc = get_field(L, "P1", &P1)))
    return rc;
  // stencil inputs: X = c2 ybar.pi, Y = c2 ybar.u, X' = c2 P4hat, Y' = c2 P3hat
  double *X = Za, *Y = Zb, *Xp = L1, *Yq = L2;
  (void)L3;
  // adjoint seeds
  if (gu_T)
    SC_CUDA(cudaMemcpyAsync(Yu, gu_T, bytes, cudaMemcpyDeviceToDevice, s));
  else
    SC_CUDA(cudaMemsetAsync(Yu, 0, bytes, s));
  if (gpi_T)
    SC_CUDA(cudaMemcpyAsync(Yp, gpi_T, bytes, cudaMemcpyDeviceToDevice, s));
  else
    SC_CUDA(cudaMemsetAsync(Yp, 0, bytes, s));
  SC_CUDA(cudaMemsetAsync(g_c2, 0, bytes, s));
  SC_CUDA(cudaMemsetAsync(D->emax_adj, 0, sizeof(unsigned) * 8 * nd, s));
  // exponent slots per adjoint step n (p = n & 1): X in 2p, Y in 2p+1,
  // X' in 4+2p, Y' in 5+2p; each slot is cleared one step ahead
  auto slot = [&](int k) { return D->emax_adj + k * nd; };
  L->launches += 2;
  SC_CUDA(dev::launch_mul(D->irects, D->ichunks, D->nichunks, c2, Yp, X,
                          fixed ? slot(0) : nullptr, D->grid_small, s));
  SC_CUDA(dev::launch_mul(D->irects, D->ichunks, D->nichunks, c2, Yu, Y,
                          fixed ? slot(1) : nullptr, D->grid_small, s));
  // Warp-specialised adjoint passes with the two-stage form, unless the
  // caller fixed the one-role kernels: the ghosts of each pass's stencil
  // inputs are gathered before it, except those of self-periodic boxes (the
  // passes read their periodic images).  Otherwise these are the only
  // gathers of the sweep and later stencil inputs have their ghosts pushed by
  // the kernels that write them.
  const bool ws = pairs && !(L->pass_fixed && !L->pass_ws);
  auto gather_ws = [&](double* f, double* g, const DChunk* list, int n) -> cudaError_t {
    if (n <= 0) return cudaSuccess;
    L->launches++;
    TimedLaunch t(q, SC_KERNEL_GATHER);
    return dev::launch_gather2(D->grects, list, n, f, g, nullptr, 0, s);
  };
  if (!ws) {
    SC_CUDA(enq_fill(q, X));
    SC_CUDA(enq_fill(q, Y));
  }

  long long n_adj = 0;
  for (int c = nck - 1; c >= 0; --c) {
    const int len = std::min(K, nsteps - c * K);
    SC_CUDA(cudaMemcpyAsync(Su, cku[c], bytes, cudaMemcpyDeviceToDevice, s));
    SC_CUDA(cudaMemcpyAsync(Sp, ckp[c], bytes, cudaMemcpyDeviceToDevice, s));
    {
      // with the warp-specialised adjoint on a level with self-periodic boxes
      // the recomputation runs the warp-specialised recording passes, which
      // need no gathers for those boxes; else the level's own pass kernels.
      // The level's choice is restored after
      bool zw = false;
      for (char w : D->box_wrap) zw = zw || (w & 2);
      const bool rec_ws = ws && (L->pass_ws || zw);
      const int pass_ws = L->pass_ws;
      if (rec_ws) L->pass_ws = 1;
      Enq qr = q;
      cudaError_t e = enq_prologue(qr, Su, pairs ? Sp : nullptr, c2, W);
      for (int n = 0; n < len && e == cudaSuccess; ++n) {
        Enq qf = qr;
        qf.push = !pairs;
        e = pairs ? enq_step_pairs(qf, Su, Sp, W, lapw.data() + 4 * n)
                  : enq_step(qf, Su, Sp, c2, W, lapw.data() + 4 * n);
      }
      L->pass_ws = pass_ws;
      SC_CUDA(e);
    }
    for (int n = len - 1; n >= 0; --n, ++n_adj) {
      const int p = (int)(n_adj & 1), pn = 1 - p;
      if (ws) {
        // first pass: (Phat4, Phat3) = L^ (X, Y); X', Y' = c2 (Phat4, Phat3);
        // the parts of ybar with Phat4, Phat3; the c2bar update.  Second pass:
        // (Phat2, Phat1) = L^ (X', Y'); ybar; X, Y = c2 (ybar.pi, ybar.u).
        // Each gather zeroes the exponent slots its pass accumulates into.
        dev::AdjWsArgs w{};
        w.items = D->items;
        w.nitems = D->nitems;
        w.ndom = nd;
        w.boxes = D->boxes;
        w.c2 = c2;
        w.yu = Yu;
        w.yp = Yp;
        w.c2bar = g_c2;
        w.q1 = lapw[4 * n + 0];
        w.q2 = lapw[4 * n + 1];
        w.q3 = lapw[4 * n + 2];
        w.q4 = lapw[4 * n + 3];
        w.coef = D->acoef;
        w.err = D->err;
        w.xg = D->xg;
        w.xg_ofs = D->xg_ofs;
        // exponent slots: the first pass writes slot 4+2p (zeroed by the
        // previous step's first pass) and zeroes 4+2pn for the next one; the
        // second writes 2pn (zeroed by the previous step's second pass) and
        // zeroes 2p, which this step's first pass has read
        SC_CUDA(gather_ws(X, Y, D->gchunks_nz, D->ngchunks_nz));
        w.z0_in = X;
        w.z1_in = Y;
        w.z0_out = Xp;
        w.z1_out = Yq;
        w.emax_in = slot(2 * p);
        w.emax_out = slot(4 + 2 * p);
        w.emax_clear = slot(4 + 2 * pn);
        L->launches++;
        {
          TimedLaunch t(q, SC_KERNEL_ADJ_A);
          SC_CUDA(dev::launch_adj_ws(false, L->arith, w, D->grid_pair_ws, s));
        }
        SC_CUDA(gather_ws(Xp, Yq, D->gchunks_nz, D->ngchunks_nz));
        w.z0_in = Xp;
        w.z1_in = Yq;
        w.z0_out = X;
        w.z1_out = Y;
        w.emax_in = slot(4 + 2 * p);
        w.emax_out = slot(2 * pn);
        w.emax_clear = slot(2 * p);
        L->launches++;
        {
          TimedLaunch t(q, SC_KERNEL_ADJ_B);
          SC_CUDA(dev::launch_adj_ws(true, L->arith, w, D->grid_pair_ws, s));
        }
        continue;
      }
      // (Phat4, Phat3) = L^ (c2 b, c2 a), (X', Y') = c2 (Phat4, Phat3)
      dev::Adj2Args a{};
      a.items = D->items_one ? D->items_one : D->items;
      a.nitems = D->items_one ? D->nitems_one : D->nitems;
      a.ndom = nd;
      a.boxes = D->boxes;
      a.c2 = c2;
      a.err = D->err;
      a.push = D->push;
      a.push_gofs = D->push_gofs;
      a.z0_in = X;
      a.z1_in = Y;
      a.p0_out = P4;
      a.p1_out = P3;
      a.z0_out = Xp;
      a.z1_out = Yq;
      a.emax_in = slot(2 * p);       // X, Y: slots 2p, 2p+1
      a.emax_out = slot(4 + 2 * p);  // X', Y': slots 4+2p, 5+2p
      a.emax_clear = slot(2 * pn);
      L->launches++;
      {
        TimedLaunch t(q, SC_KERNEL_ADJ_A);
        SC_CUDA(dev::launch_adj2(false, L->arith, a, D->grid_pair, s));
      }
      // (Phat2, Phat1) = L^ (X', Y')
      a.z0_in = Xp;
      a.z1_in = Yq;
      a.p0_out = P2;
      a.p1_out = P1;
      a.z0_out = a.z1_out = nullptr;
      a.emax_in = slot(4 + 2 * p);
      a.emax_out = nullptr;
      a.emax_clear = slot(4 + 2 * pn);
      L->launches++;
      {
        TimedLaunch t(q, SC_KERNEL_ADJ_B);
        SC_CUDA(dev::launch_adj2(true, L->arith, a, D->grid_pair, s));
      }
      // the combination, pointwise
      dev::AdjCombineArgs b{};
      b.yu = Yu;
      b.yp = Yp;
      b.p4 = P4;
      b.p3 = P3;
      b.p2 = P2;
      b.p1 = P1;
      b.q1 = lapw[4 * n + 0];
      b.q2 = lapw[4 * n + 1];
      b.q3 = lapw[4 * n + 2];
      b.q4 = lapw[4 * n + 3];
      b.c2 = c2;
      b.c2bar = g_c2;
      b.x_out = X;
      b.y_out = Y;
      b.coef = D->acoef;
      b.boxes = D->boxes;
      b.push = D->push;
      b.push_gofs = D->push_gofs;
      b.emax_x = slot(2 * pn);
      b.emax_y = slot(2 * pn + 1);
      L->launches++;
      {
        TimedLaunch t(q, SC_KERNEL_ADJ_C);
        SC_CUDA(dev::launch_adj_combine(L->arith, D->irects, D->pchunks, D->npchunks, b,
                                        D->grid_small, s));
      }
    }
  }
  SC_CUDA(cudaMemcpyAsync(g_u0, Yu, bytes, cudaMemcpyDeviceToDevice, s));
  SC_CUDA(cudaMemcpyAsync(g_pi0, Yp, bytes, cudaMemcpyDeviceToDevice, s));
  return SC_OK;
}

int sc_level_grad(sc_level* L, const double* u0, const double* pi0, const double* c2,
                  const double* dt, int32_t ndt, int32_t nsteps, int32_t ckpt_every,
                  const double* gu_T, const double* gpi_T, double* g_u0, double* g_pi0,
                  double* g_c2, double* u_T, double* pi_T, void* stream) {
  int rc = sc_level_forward_tape(L, u0, pi0, c2, dt, ndt, nsteps, ckpt_every, u_T, pi_T,
                                 stream);
  if (rc) return rc;
  return sc_level_backward_tape(L, c2, gu_T, gpi_T, g_u0, g_pi0, g_c2, stream);
}

int sc_level_set_pass_kernel(sc_level* L, int32_t kind) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (kind != SC_PASS_ONE_ROLE && kind != SC_PASS_WARP_SPECIALISED)
    return set_error(SC_EINVAL, "kind must be SC_PASS_ONE_ROLE or SC_PASS_WARP_SPECIALISED");
  L->pass_ws = kind;  // the step graphs are keyed by it
  L->pass_fixed = true;
  return SC_OK;
}

int sc_level_get_pass_kernel(const sc_level* L, int32_t* kind) {
  if (!L || !kind) return set_error(SC_EINVAL, "NULL argument");
  *kind = L->pass_ws;
  return SC_OK;
}

int sc_level_arm_wait_test(sc_level* L) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!L->pass_ws || L->fuse != 2)
    return set_error(SC_EINVAL, "the wait test needs the warp-specialised two-stage passes");
  L->wait_test = 1;
  return SC_OK;
}

int sc_level_kernel_time(sc_level* L, int32_t kind, double* ms, int64_t* launches) {
  if (!L || !ms || !launches) return set_error(SC_EINVAL, "NULL argument");
  *ms = 0.0;
  *launches = 0;
  DeviceState* D = L->dev;
  if (!D) return SC_OK;
  for (size_t i = 0; i < D->ev_used; ++i) {
    if (D->ev_kind[i] != kind) continue;
    SC_CUDA(cudaEventSynchronize(D->ev_pool[i].second));
    float t = 0.f;
    SC_CUDA(cudaEventElapsedTime(&t, D->ev_pool[i].first, D->ev_pool[i].second));
    *ms += t;
    ++*launches;
  }
  return SC_OK;
}

int sc_level_kernel_times(sc_level* L, double* stage_ms, int64_t* stage_launches,
                          double* gather_ms, int64_t* gather_launches) {
  int rc = sc_level_kernel_time(L, SC_KERNEL_STAGE, stage_ms, stage_launches);
  if (rc) return rc;
  return sc_level_kernel_time(L, SC_KERNEL_GATHER, gather_ms, gather_launches);
}

int sc_level_set_profiling(sc_level* L, int32_t on) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  L->profile = on ? 1 : 0;
  return SC_OK;
}

int sc_level_set_tuning(sc_level* L, int32_t cls, const sc_tile* t, int32_t ctas_per_sm) {
  if (!L || !t) return set_error(SC_EINVAL, "NULL argument");
  if (cls < 0 || cls >= (int32_t)L->classes.size()) return set_error(SC_EINVAL, "bad class");
  const int tx = t->tile_x;
  if (tx != 16 && tx != 32 && tx != 64)
    return set_error(SC_EINVAL, "tile_x must be 16, 32 or 64");
  if ((tx / 2) * t->tile_y != dev::stage_threads())
    return set_error(SC_EINVAL, "tile_x/2 * tile_y must equal 256");
  if (t->tile_z < 1) return set_error(SC_EINVAL, "tile_z must be >= 1");
  if (ctas_per_sm < 0 || ctas_per_sm > 8) return set_error(SC_EINVAL, "ctas_per_sm in [0, 8]");
  L->classes[cls].tile = *t;
  L->classes[cls].tile.reserved = 0;
  L->classes[cls].fixed = true;
  L->classes[cls].has_one = false;  // an explicit tile serves every kernel
  if (ctas_per_sm > 0) L->ctas_per_sm = ctas_per_sm;
  if (L->dev) return upload_items(L);
  return SC_OK;
}

}  // extern "C"
