// Host-only part of the C ABI: level construction and validation with the
// bboxset algebra, the level layout, the ghost-exchange list, size classes,
// and the bboxset entry points.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/sc_bboxset.h"
#include "../../include/sc_dist.h"
#include "../../include/sc_level.h"
#include "bboxset.hpp"
#include "level.hpp"

namespace sc {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

void release_device(sc_level* L);  // runtime.cu

static BBox3 to_box(const int64_t* lo, const int64_t* hi) {
  BBox3 b;
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = lo[d];
    b.hi[d] = hi[d];
  }
  return b;
}

static int64_t roundup(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

// Ghost region of one box: the star-shaped shell
// (union_d expand_d(box, g)) minus the box.
static BBoxSet3 star_shell(const BBox3& b, int g) {
  BBoxSet3 B = BBoxSet3::box(b);
  BBoxSet3 u;
  for (int d = 0; d < 3; ++d) {
    int64_t lo_by[3] = {0, 0, 0}, hi_by[3] = {0, 0, 0};
    lo_by[d] = hi_by[d] = g;
    u = u | B.expanded(lo_by, hi_by);
  }
  return u - B;
}

// The exchange list: for every box b and every box o of the same domain and
// every periodic image s, the rectangles of shell(b) & shift(o, s * L), each
// copied from o's interior point p - s * L (the communication schedule the
// paper derives from bboxset intersections, Sec. 2).
static void build_exchange(sc_level* L) {
  const int nb = (int)L->boxes.size();
  L->copies.clear();
  for (int b = 0; b < nb; ++b) {
    const sc_box& B = L->boxes[b];
    const sc_domain& D = L->doms[B.domain];
    const BBox3 bb = to_box(B.lo, B.hi);
    const BBoxSet3 shell = star_shell(bb, 2);
    BBox3 reach = bb;
    for (int d = 0; d < 3; ++d) {
      reach.lo[d] -= 2;
      reach.hi[d] += 2;
    }
    int64_t len[3];
    for (int d = 0; d < 3; ++d) len[d] = D.hi[d] - D.lo[d];
    for (int o = 0; o < nb; ++o) {
      const sc_box& O = L->boxes[o];
      if (O.domain != B.domain) continue;
      for (int sz = -1; sz <= 1; ++sz)
        for (int sy = -1; sy <= 1; ++sy)
          for (int sx = -1; sx <= 1; ++sx) {
            const int s[3] = {sx, sy, sz};
            bool ok = true;
            for (int d = 0; d < 3; ++d)
              if (s[d] != 0 && !(D.periodic & (1u << d))) ok = false;
            if (!ok) continue;
            int64_t v[3];
            BBox3 ob = to_box(O.lo, O.hi);
            for (int d = 0; d < 3; ++d) {
              v[d] = s[d] * len[d];
              ob.lo[d] += v[d];
              ob.hi[d] += v[d];
            }
            // bounding-box test before the set intersection
            bool overlap = true;
            for (int d = 0; d < 3; ++d)
              if (ob.hi[d] <= reach.lo[d] || ob.lo[d] >= reach.hi[d]) overlap = false;
            if (!overlap) continue;
            const BBoxSet3 I = shell & BBoxSet3::box(ob);
            for (const BBox3& r : I.boxes()) {
              sc_copy c;
              c.src_box = o;
              c.dst_box = b;
              for (int d = 0; d < 3; ++d) {
                c.dst_lo[d] = r.lo[d];
                c.src_lo[d] = r.lo[d] - v[d];
                c.ext[d] = r.hi[d] - r.lo[d];
              }
              L->copies.push_back(c);
            }
          }
    }
  }
}

// 32 x 16 tiles unless the box is at most 16 wide (measured on the uneven
// 64-box level with the warp-specialised passes: 29.6 G updates/s with 32 x 16
// tiles, 25.5 G with 64 x 8; the autotuner moves from here)
static sc_tile default_tile(const std::array<int64_t, 3>& ext) {
  sc_tile t{};
  const int64_t nx = ext[0];
  t.tile_x = nx <= 16 ? 16 : 32;
  t.tile_y = 2 * 256 / t.tile_x;
  t.tile_z = 32;
  return t;
}

static void build_classes(sc_level* L) {
  L->classes.clear();
  L->box_class.assign(L->boxes.size(), 0);
  std::map<std::array<int64_t, 3>, int> idx;
  for (size_t b = 0; b < L->boxes.size(); ++b) {
    std::array<int64_t, 3> e;
    for (int d = 0; d < 3; ++d) e[d] = roundup(L->boxes[b].hi[d] - L->boxes[b].lo[d], 8);
    auto it = idx.find(e);
    if (it == idx.end()) {
      it = idx.emplace(e, (int)L->classes.size()).first;
      L->classes.push_back(SizeClass{e, default_tile(e)});
    }
    L->box_class[b] = it->second;
  }
}

static int validate(const sc_box* boxes, int32_t nboxes, const sc_domain* doms,
                    int32_t ndoms) {
  if (nboxes <= 0 || !boxes) return set_error(SC_EINVAL, "level needs at least one box");
  if (ndoms <= 0 || !doms) return set_error(SC_EINVAL, "level needs at least one domain");
  for (int32_t d = 0; d < ndoms; ++d) {
    const sc_domain& D = doms[d];
    if (!(D.h > 0.0)) return set_error(SC_EINVAL, "domain " + std::to_string(d) + ": h <= 0");
    if (D.reserved != 0 || (D.periodic & ~7u))
      return set_error(SC_EINVAL, "domain " + std::to_string(d) + ": reserved bits set");
    for (int a = 0; a < 3; ++a)
      if (D.hi[a] - D.lo[a] < 2)
        return set_error(SC_EINVAL, "domain " + std::to_string(d) + ": extent < 2");
  }
  std::vector<std::vector<int>> per(ndoms);
  for (int32_t b = 0; b < nboxes; ++b) {
    const sc_box& B = boxes[b];
    const std::string nm = "box " + std::to_string(b);
    if (B.domain < 0 || B.domain >= ndoms) return set_error(SC_EINVAL, nm + ": bad domain");
    if (B.reserved != 0) return set_error(SC_EINVAL, nm + ": reserved field set");
    const sc_domain& D = doms[B.domain];
    for (int a = 0; a < 3; ++a) {
      if (B.hi[a] - B.lo[a] < 2) return set_error(SC_EINVAL, nm + ": edge < 2");
      if (B.hi[a] - B.lo[a] > (1 << 24)) return set_error(SC_EINVAL, nm + ": edge too large");
      if (B.lo[a] < D.lo[a] || B.hi[a] > D.hi[a])
        return set_error(SC_EINVAL, nm + ": not inside its domain");
    }
    per[B.domain].push_back(b);
  }
  // each domain is tiled exactly: union == domain and no overlap
  for (int32_t d = 0; d < ndoms; ++d) {
    const sc_domain& D = doms[d];
    if (per[d].empty()) return set_error(SC_EINVAL, "domain " + std::to_string(d) + " has no box");
    BBoxSet3 u;
    int64_t total = 0;
    for (int b : per[d]) {
      const BBoxSet3 s = BBoxSet3::box(boxes[b].lo, boxes[b].hi);
      const BBoxSet3 common = u & s;
      if (!common.empty())
        return set_error(SC_EINVAL, "box " + std::to_string(b) + " overlaps another box of domain " +
                                        std::to_string(d));
      u = u | s;
      total += s.size();
    }
    const BBoxSet3 dom = BBoxSet3::box(D.lo, D.hi);
    if (u != dom)
      return set_error(SC_EINVAL, "boxes of domain " + std::to_string(d) + " do not tile it");
    (void)total;
  }
  return SC_OK;
}

// Layout, exchange list and size classes of a level whose boxes and domains
// are set (every box stored, box-major; the exchange among those boxes).
static int build_level(sc_level* L) {
  L->all_periodic = true;
  for (const auto& D : L->doms)
    if (D.periodic != 7u) L->all_periodic = false;
  // layout: interior corner of every box on a 16-double (128-byte) line
  int64_t base = 14;
  for (const auto& B : L->boxes) {
    const int64_t nx = B.hi[0] - B.lo[0], ny = B.hi[1] - B.lo[1], nz = B.hi[2] - B.lo[2];
    const int64_t py = roundup(nx + 4, 16), pz = py * (ny + 4), st = pz * (nz + 4);
    L->py.push_back(py);
    L->pz.push_back(pz);
    L->storage.push_back(st);
    L->off.push_back(base + 2 + 2 * py + 2 * pz);
    base += st;
  }
  L->field_size = base + 2;
  if (L->field_size >= (int64_t(1) << 31))
    return set_error(SC_EINVAL, "level too large: a field must hold fewer than 2^31 doubles");
  build_exchange(L);
  build_classes(L);
  sc::plan_xface_reads(L);
  return SC_OK;
}

static int64_t box_points(const sc_box& B) {
  return (B.hi[0] - B.lo[0]) * (B.hi[1] - B.lo[1]) * (B.hi[2] - B.lo[2]);
}

// Greedy balance by point count: boxes in decreasing size (ties: lower
// index first) each go to the rank with the fewest points so far (ties:
// lower rank).  The largest load then exceeds the mean by less than the
// largest box.
static void partition_greedy(const sc_box* boxes, int nb, int nranks, int32_t* rank_of) {
  std::vector<int> order(nb);
  for (int b = 0; b < nb; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return box_points(boxes[a]) > box_points(boxes[b]);
  });
  std::vector<int64_t> load(nranks, 0);
  for (int b : order) {
    int r = 0;
    for (int k = 1; k < nranks; ++k)
      if (load[k] < load[r]) r = k;
    rank_of[b] = r;
    load[r] += box_points(boxes[b]);
  }
}

// Recursive bisection in space: the boxes of a group of ranks are ordered
// by their centres along the longest axis of the group's bounding box and
// cut where the lower part's share of the points comes closest to its
// share of the ranks (each part keeping at least as many boxes as ranks);
// then each part is split again.  Boxes that are near each other share a
// rank, so fewer ghost copies cross ranks than with the greedy split.
static void partition_bisect(const sc_box* boxes, std::vector<int> group, int r0, int nr,
                             int32_t* rank_of) {
  if (nr == 1) {
    for (int b : group) rank_of[b] = r0;
    return;
  }
  int64_t lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = INT64_MAX;
    hi[d] = INT64_MIN;
  }
  for (int b : group)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], boxes[b].lo[d]);
      hi[d] = std::max(hi[d], boxes[b].hi[d]);
    }
  int axis = 0;
  for (int d = 1; d < 3; ++d)
    if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
  std::stable_sort(group.begin(), group.end(), [&](int a, int b) {
    return boxes[a].lo[axis] + boxes[a].hi[axis] < boxes[b].lo[axis] + boxes[b].hi[axis];
  });
  const int nl = nr / 2;
  int64_t total = 0;
  for (int b : group) total += box_points(boxes[b]);
  // cut after k boxes, nl <= k <= size - (nr - nl)
  int best = nl;
  double best_gap = -1.0;
  int64_t acc = 0;
  const int n = (int)group.size();
  for (int k = 1; k <= n - (nr - nl); ++k) {
    acc += box_points(boxes[group[k - 1]]);
    if (k < nl) continue;
    const double gap = std::fabs((double)acc / (double)total - (double)nl / (double)nr);
    if (best_gap < 0.0 || gap < best_gap) {
      best_gap = gap;
      best = k;
    }
  }
  partition_bisect(boxes, std::vector<int>(group.begin(), group.begin() + best), r0, nl,
                   rank_of);
  partition_bisect(boxes, std::vector<int>(group.begin() + best, group.end()), r0 + nl,
                   nr - nl, rank_of);
}

}  // namespace sc

using namespace sc;

extern "C" {

const char* sc_last_error(void) { return g_last_error.c_str(); }

int sc_level_create(const sc_box* boxes, int32_t nboxes, const sc_domain* doms, int32_t ndoms,
                    int32_t ghost, sc_level** out) {
  if (!out) return set_error(SC_EINVAL, "out is NULL");
  *out = nullptr;
  if (ghost != 2) return set_error(SC_EINVAL, "ghost width must be 2");
  int rc = validate(boxes, nboxes, doms, ndoms);
  if (rc) return rc;
  sc_level* L = new (std::nothrow) sc_level();
  if (!L) return set_error(SC_ENOMEM, "out of host memory");
  try {
    L->boxes.assign(boxes, boxes + nboxes);
    L->doms.assign(doms, doms + ndoms);
    rc = build_level(L);
  } catch (const std::bad_alloc&) {
    rc = set_error(SC_ENOMEM, "out of host memory");
  }
  if (rc) {
    delete L;
    return rc;
  }
  *out = L;
  return SC_OK;
}

void sc_level_destroy(sc_level* L) {
  if (!L) return;
  release_device(L);
  delete L;
}

int sc_level_field_size(const sc_level* L, int64_t* n) {
  if (!L || !n) return set_error(SC_EINVAL, "NULL argument");
  *n = L->field_size;
  return SC_OK;
}

int sc_level_num_boxes(const sc_level* L, int32_t* n) {
  if (!L || !n) return set_error(SC_EINVAL, "NULL argument");
  *n = (int32_t)L->boxes.size();
  return SC_OK;
}

int sc_level_box_layout(const sc_level* L, int32_t b, int64_t* offset, int64_t dims[3],
                        int64_t pitch[3]) {
  if (!L || !offset || !dims || !pitch) return set_error(SC_EINVAL, "NULL argument");
  if (b < 0 || b >= (int32_t)L->boxes.size()) return set_error(SC_EINVAL, "box out of range");
  *offset = L->off[b];
  for (int d = 0; d < 3; ++d) dims[d] = L->boxes[b].hi[d] - L->boxes[b].lo[d];
  pitch[0] = 1;
  pitch[1] = L->py[b];
  pitch[2] = L->pz[b];
  return SC_OK;
}

int sc_level_exchange_list(const sc_level* L, sc_copy* out, int64_t cap, int64_t* n) {
  if (!L || !n) return set_error(SC_EINVAL, "NULL argument");
  if (cap > 0 && !out) return set_error(SC_EINVAL, "out is NULL");
  *n = (int64_t)L->copies.size();
  const int64_t m = std::min<int64_t>(cap, *n);
  if (m > 0) std::memcpy(out, L->copies.data(), (size_t)m * sizeof(sc_copy));
  return SC_OK;
}

int sc_level_size_classes(const sc_level* L, int32_t* nclasses, int32_t* class_of_box) {
  if (!L || !nclasses) return set_error(SC_EINVAL, "NULL argument");
  *nclasses = (int32_t)L->classes.size();
  if (class_of_box)
    for (size_t b = 0; b < L->boxes.size(); ++b) class_of_box[b] = L->box_class[b];
  return SC_OK;
}

int sc_level_set_arith(sc_level* L, int32_t arith) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (arith != SC_ARITH_FP64 && arith != SC_ARITH_FIXED)
    return set_error(SC_EINVAL, "unknown arithmetic");
  if (L->arith == arith) return SC_OK;
  L->arith = arith;
  if (L->dev) return upload_items(L);  // occupancy (grid) depends on the arithmetic
  return SC_OK;
}

int sc_level_set_fusion(sc_level* L, int32_t stages_per_pass) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (stages_per_pass != 1 && stages_per_pass != 2)
    return set_error(SC_EINVAL, "stages_per_pass must be 1 or 2");
  L->fuse = stages_per_pass;  // the step graphs are keyed by it
  L->fuse_fixed = true;
  return SC_OK;
}

int sc_level_get_fusion(const sc_level* L, int32_t* stages_per_pass) {
  if (!L || !stages_per_pass) return set_error(SC_EINVAL, "NULL argument");
  *stages_per_pass = L->fuse;
  return SC_OK;
}

int sc_level_set_staging(sc_level* L, int32_t staging) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (staging != SC_STAGING_REGISTERS && staging != SC_STAGING_SHARED)
    return set_error(SC_EINVAL, "staging must be SC_STAGING_REGISTERS or SC_STAGING_SHARED");
  L->staging = staging;  // the step graphs are keyed by it
  L->staging_fixed = true;
  return SC_OK;
}

int sc_level_get_staging(const sc_level* L, int32_t* staging) {
  if (!L || !staging) return set_error(SC_EINVAL, "NULL argument");
  *staging = L->staging;
  return SC_OK;
}

int sc_level_get_tuning(const sc_level* L, int32_t size_class, sc_tile* tile) {
  if (!L || !tile) return set_error(SC_EINVAL, "NULL argument");
  if (size_class < 0 || size_class >= (int32_t)L->classes.size())
    return set_error(SC_EINVAL, "bad class");
  *tile = L->classes[size_class].tile;
  return SC_OK;
}

int sc_level_launch_count(const sc_level* L, int64_t* n) {
  if (!L || !n) return set_error(SC_EINVAL, "NULL argument");
  *n = L->launches;
  return SC_OK;
}

// ---- bboxset entry points ------------------------------------------------

static int read_set(const int64_t* a, int64_t na, BBoxSet3* s) {
  if (na < 0 || (na > 0 && !a)) return set_error(SC_EINVAL, "bad box array");
  BBoxSet3 r;
  for (int64_t i = 0; i < na; ++i) {
    for (int d = 0; d < 3; ++d)
      if (a[6 * i + d] > a[6 * i + 3 + d]) return set_error(SC_EINVAL, "box with lo > hi");
    r = r | BBoxSet3::box(a + 6 * i, a + 6 * i + 3);
  }
  *s = std::move(r);
  return SC_OK;
}

static int write_boxes(const BBoxSet3& s, int64_t* out, int64_t cap, int64_t* n) {
  const std::vector<BBox3> bs = s.boxes();
  *n = (int64_t)bs.size();
  if (cap > 0 && !out) return set_error(SC_EINVAL, "out is NULL");
  for (int64_t i = 0; i < std::min<int64_t>(cap, *n); ++i)
    for (int d = 0; d < 3; ++d) {
      out[6 * i + d] = bs[i].lo[d];
      out[6 * i + 3 + d] = bs[i].hi[d];
    }
  return SC_OK;
}

int sc_bboxset_op(int32_t op, const int64_t* a, int64_t na, const int64_t* b, int64_t nb,
                  int64_t* out, int64_t cap, int64_t* n) {
  if (!n) return set_error(SC_EINVAL, "n is NULL");
  BBoxSet3 A, B;
  int rc = read_set(a, na, &A);
  if (rc) return rc;
  rc = read_set(b, nb, &B);
  if (rc) return rc;
  SetOp o;
  switch (op) {
    case SC_SET_UNION: o = SetOp::Union; break;
    case SC_SET_INTERSECTION: o = SetOp::Intersection; break;
    case SC_SET_DIFFERENCE: o = SetOp::Difference; break;
    case SC_SET_XOR: o = SetOp::Xor; break;
    default: return set_error(SC_EINVAL, "unknown set operation");
  }
  return write_boxes(BBoxSet3::binop(A, B, o), out, cap, n);
}

int sc_bboxset_derivative(const int64_t* a, int64_t na, int64_t* pts, int64_t cap, int64_t* n) {
  if (!n) return set_error(SC_EINVAL, "n is NULL");
  BBoxSet3 A;
  int rc = read_set(a, na, &A);
  if (rc) return rc;
  std::vector<std::array<int64_t, 3>> p;
  A.derivative_points(p);
  *n = (int64_t)p.size();
  if (cap > 0 && !pts) return set_error(SC_EINVAL, "pts is NULL");
  for (int64_t i = 0; i < std::min<int64_t>(cap, *n); ++i)
    for (int d = 0; d < 3; ++d) pts[3 * i + d] = p[i][d];
  return SC_OK;
}

int sc_bboxset_expand_shift(const int64_t* a, int64_t na, const int64_t lo_by[3],
                            const int64_t hi_by[3], const int64_t v[3], int64_t* out,
                            int64_t cap, int64_t* n) {
  if (!n || !lo_by || !hi_by || !v) return set_error(SC_EINVAL, "NULL argument");
  for (int d = 0; d < 3; ++d)
    if (lo_by[d] < 0 || hi_by[d] < 0) return set_error(SC_EINVAL, "negative expansion");
  BBoxSet3 A;
  int rc = read_set(a, na, &A);
  if (rc) return rc;
  return write_boxes(A.expanded(lo_by, hi_by).shifted(v), out, cap, n);
}

int sc_bboxset_coarsen(const int64_t* a, int64_t na, int64_t ratio, int64_t* out, int64_t cap,
                       int64_t* n) {
  if (!n) return set_error(SC_EINVAL, "NULL argument");
  if (ratio < 1) return set_error(SC_EINVAL, "ratio must be >= 1");
  BBoxSet3 A;
  int rc = read_set(a, na, &A);
  if (rc) return rc;
  return write_boxes(coarsened(A, ratio), out, cap, n);
}

int sc_bboxset_size(const int64_t* a, int64_t na, int64_t* npoints) {
  if (!npoints) return set_error(SC_EINVAL, "NULL argument");
  BBoxSet3 A;
  int rc = read_set(a, na, &A);
  if (rc) return rc;
  *npoints = A.size();
  return SC_OK;
}

// ---- distributed level ---------------------------------------------------

int sc_dist_partition(const sc_box* boxes, int32_t nboxes, int32_t nranks, int32_t method,
                      int32_t* rank_of_box) {
  if (!boxes || !rank_of_box) return set_error(SC_EINVAL, "NULL argument");
  if (nranks < 1) return set_error(SC_EINVAL, "nranks must be >= 1");
  if (nboxes < nranks) return set_error(SC_EINVAL, "fewer boxes than ranks");
  try {
    if (method == SC_DIST_GREEDY) {
      partition_greedy(boxes, nboxes, nranks, rank_of_box);
    } else if (method == SC_DIST_BISECT) {
      std::vector<int> all(nboxes);
      for (int b = 0; b < nboxes; ++b) all[b] = b;
      partition_bisect(boxes, all, 0, nranks, rank_of_box);
    } else {
      return set_error(SC_EINVAL, "unknown partition method");
    }
  } catch (const std::bad_alloc&) {
    return set_error(SC_ENOMEM, "out of host memory");
  }
  return SC_OK;
}

int sc_dist_create(const sc_box* boxes, int32_t nboxes, const sc_domain* doms, int32_t ndoms,
                   int32_t ghost, const int32_t* rank_of_box, int32_t nranks, int32_t rank,
                   sc_level** out) {
  if (!out) return set_error(SC_EINVAL, "out is NULL");
  *out = nullptr;
  if (ghost != 2) return set_error(SC_EINVAL, "ghost width must be 2");
  if (!rank_of_box) return set_error(SC_EINVAL, "rank_of_box is NULL");
  if (nranks < 1 || rank < 0 || rank >= nranks) return set_error(SC_EINVAL, "bad rank");
  int rc = validate(boxes, nboxes, doms, ndoms);
  if (rc) return rc;
  for (int32_t d = 0; d < ndoms; ++d)
    if (doms[d].periodic != 7u)
      return set_error(SC_EINVAL, "a distributed level needs domains periodic on every axis");
  std::vector<int> owned(nranks, 0);
  for (int32_t b = 0; b < nboxes; ++b) {
    if (rank_of_box[b] < 0 || rank_of_box[b] >= nranks)
      return set_error(SC_EINVAL, "box " + std::to_string(b) + ": rank out of range");
    owned[rank_of_box[b]]++;
  }
  for (int r = 0; r < nranks; ++r)
    if (!owned[r]) return set_error(SC_EINVAL, "rank " + std::to_string(r) + " owns no box");
  sc_level* L = new (std::nothrow) sc_level();
  if (!L) return set_error(SC_ENOMEM, "out of host memory");
  try {
    // the whole level's exchange list, in its deterministic order: every
    // rank computes the same list, so the two ends of each peer pair filter
    // the same copies in the same order
    sc_level whole;
    whole.boxes.assign(boxes, boxes + nboxes);
    whole.doms.assign(doms, doms + ndoms);
    build_exchange(&whole);
    std::vector<int> local(nboxes, -1);
    for (int32_t b = 0; b < nboxes; ++b)
      if (rank_of_box[b] == rank) {
        local[b] = (int)L->boxes.size();
        L->boxes.push_back(boxes[b]);
        L->global_box.push_back(b);
      }
    L->doms.assign(doms, doms + ndoms);
    L->partial = true;
    L->rank = rank;
    L->nranks = nranks;
    L->fuse = 2;  // the exchange sits between the two passes of a step
    L->fuse_fixed = true;
    rc = build_level(L);  // layout and the exchange among this rank's boxes
    if (!rc) {
      std::map<int, PeerLists> per;
      for (const sc_copy& c : whole.copies) {
        const int rs = rank_of_box[c.src_box], rd = rank_of_box[c.dst_box];
        if (rs == rd) continue;
        if (rd == rank) {
          sc_copy e = c;
          e.dst_box = local[c.dst_box];
          PeerLists& P = per[rs];
          P.recv.push_back(e);
          P.recv_points += c.ext[0] * c.ext[1] * c.ext[2];
        } else if (rs == rank) {
          sc_copy e = c;
          e.src_box = local[c.src_box];
          PeerLists& P = per[rd];
          P.send.push_back(e);
          P.send_points += c.ext[0] * c.ext[1] * c.ext[2];
        }
      }
      int64_t so = 0, ro = 0;
      for (auto& kv : per) {
        kv.second.peer = kv.first;
        kv.second.send_offset = so;
        kv.second.recv_offset = ro;
        so += 2 * kv.second.send_points;
        ro += 2 * kv.second.recv_points;
        L->peers.push_back(kv.second);
      }
      L->send_doubles = so;
      L->recv_doubles = ro;
      if (so >= (int64_t(1) << 31) || ro >= (int64_t(1) << 31))
        rc = set_error(SC_EINVAL, "exchange buffer too large");
    }
  } catch (const std::bad_alloc&) {
    rc = set_error(SC_ENOMEM, "out of host memory");
  }
  if (rc) {
    delete L;
    return rc;
  }
  *out = L;
  return SC_OK;
}

int sc_dist_info(const sc_level* L, int32_t* rank, int32_t* nranks, int32_t* npeers) {
  if (!L || !rank || !nranks || !npeers) return set_error(SC_EINVAL, "NULL argument");
  *rank = L->rank;
  *nranks = L->nranks;
  *npeers = (int32_t)L->peers.size();
  return SC_OK;
}

int sc_dist_global_box(const sc_level* L, int32_t box, int32_t* global_box) {
  if (!L || !global_box) return set_error(SC_EINVAL, "NULL argument");
  if (box < 0 || box >= (int32_t)L->boxes.size()) return set_error(SC_EINVAL, "box out of range");
  *global_box = L->partial ? L->global_box[box] : box;
  return SC_OK;
}

int sc_dist_buffer_sizes(const sc_level* L, int64_t* send_doubles, int64_t* recv_doubles) {
  if (!L || !send_doubles || !recv_doubles) return set_error(SC_EINVAL, "NULL argument");
  *send_doubles = L->send_doubles;
  *recv_doubles = L->recv_doubles;
  return SC_OK;
}

int sc_dist_peer(const sc_level* L, int32_t i, int32_t* peer, int64_t* send_points,
                 int64_t* recv_points, int64_t* send_offset, int64_t* recv_offset) {
  if (!L || !peer || !send_points || !recv_points || !send_offset || !recv_offset)
    return set_error(SC_EINVAL, "NULL argument");
  if (i < 0 || i >= (int32_t)L->peers.size()) return set_error(SC_EINVAL, "peer out of range");
  const PeerLists& P = L->peers[i];
  *peer = P.peer;
  *send_points = P.send_points;
  *recv_points = P.recv_points;
  *send_offset = P.send_offset;
  *recv_offset = P.recv_offset;
  return SC_OK;
}

int sc_dist_list(const sc_level* L, int32_t i, int32_t recv, sc_copy* out, int64_t cap,
                 int64_t* n) {
  if (!L || !n) return set_error(SC_EINVAL, "NULL argument");
  if (i < 0 || i >= (int32_t)L->peers.size()) return set_error(SC_EINVAL, "peer out of range");
  if (cap > 0 && !out) return set_error(SC_EINVAL, "out is NULL");
  const std::vector<sc_copy>& v = recv ? L->peers[i].recv : L->peers[i].send;
  *n = (int64_t)v.size();
  const int64_t m = std::min<int64_t>(cap, *n);
  if (m > 0) std::memcpy(out, v.data(), (size_t)m * sizeof(sc_copy));
  return SC_OK;
}

}  // extern "C"
