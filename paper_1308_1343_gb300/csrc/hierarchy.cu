// Two-level refinement hierarchy: the prolongation and restriction lists
// derived with the bboxset algebra (arXiv 1308.1343, Sec. 2: AMR operators
// determined from bboxsets), their kernels' launches, and the Berger-Oliger
// step.  The readings (operators, buffer zone, sub-cycling) are stated in
// include/sc_hierarchy.h.
#include <algorithm>
#include <cstdint>
#include <array>
#include <string>
#include <vector>

#include "../../include/sc_hierarchy.h"
#include "bboxset.hpp"
#include "level.hpp"

using sc::BBox3;
using sc::BBoxSet3;

struct sc_hierarchy {
  sc_level* coarse = nullptr;
  sc_level* fine = nullptr;
  int buffer = 4;
  BBox3 R, T;
  std::vector<sc::dev::DProl> prol;
  std::vector<sc::dev::DChunk> prol_chunks;
  // per coarse box, the bounding box of the prolongation stencils' coarse
  // points: where time interpolation is needed
  std::vector<sc::dev::DRect> blend;
  std::vector<sc::dev::DChunk> blend_chunks;
  std::vector<sc::dev::DRestr> restr;
  std::vector<sc::dev::DChunk> restr_chunks;
  // each list's rectangles in level coordinates (lo, hi), for the queries
  std::vector<std::array<int64_t, 6>> prol_rects, restr_rects;
  int64_t n_prol = 0, n_restr = 0;
  // device copies (on the coarse level's device)
  sc::dev::DProl* d_prol = nullptr;
  sc::dev::DChunk* d_prol_chunks = nullptr;
  sc::dev::DRect* d_blend = nullptr;
  sc::dev::DChunk* d_blend_chunks = nullptr;
  sc::dev::DRestr* d_restr = nullptr;
  sc::dev::DChunk* d_restr_chunks = nullptr;
  int device = -1;
};

namespace sc {
namespace {

BBox3 box_of(const int64_t* lo, const int64_t* hi) {
  BBox3 b;
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = lo[d];
    b.hi[d] = hi[d];
  }
  return b;
}

// Star-shaped ghost shell of a box: points outside along exactly one axis,
// within 2 of it.
BBoxSet3 star_shell(const BBox3& b) {
  const BBoxSet3 B = BBoxSet3::box(b);
  BBoxSet3 s;
  for (int d = 0; d < 3; ++d) {
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    lo[d] = hi[d] = 2;
    s = s | B.expanded(lo, hi);
  }
  return s - B;
}

// Element index of level point p in box b's padded layout.
long long elem(const sc_level* L, int b, const int64_t* p) {
  const sc_box& B = L->boxes[b];
  return (long long)(L->off[b] + (p[0] - B.lo[0]) + (p[1] - B.lo[1]) * L->py[b] +
                     (p[2] - B.lo[2]) * L->pz[b]);
}

// Fine points whose prolongation stencil lies inside coarse box [clo, chi):
// along each axis, odd f needs coarse (f-3)/2 .. (f+3)/2 and even f needs f/2,
// so f in [2 clo + 3, 2 chi - 4) always fits (a conservative box).
BBox3 safe_fine(const sc_box& cb) {
  BBox3 r;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = 2 * cb.lo[d] + 3;
    r.hi[d] = 2 * cb.hi[d] - 4;
  }
  return r;
}

void add_chunks(int rect, int64_t n, std::vector<dev::DChunk>& out,
                int chunk = dev::kGatherChunk) {
  for (int64_t f = 0; f < n; f += chunk) out.push_back(dev::DChunk{rect, (int)f});
}

// First coarse index of fine index f's stencil, and one past its last.
int64_t stencil_lo(int64_t f) { return (f & 1) ? (f - 3) / 2 : f / 2; }
int64_t stencil_hi(int64_t f) { return (f & 1) ? (f + 3) / 2 + 1 : f / 2 + 1; }

template <class T>
int upload(T** dst, const std::vector<T>& v) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (v.empty()) return SC_OK;
  if (cudaMalloc(dst, v.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(SC_ENOMEM, "hierarchy: device allocation failed");
  }
  if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(SC_ECUDA, "hierarchy: upload failed");
  return SC_OK;
}

int check_lists(const sc_hierarchy* H);

int build_lists(sc_hierarchy* H) {
  const sc_level* C = H->coarse;
  const sc_level* F = H->fine;
  const BBoxSet3 Rs = BBoxSet3::box(H->R), Ts = BBoxSet3::box(H->T);
  std::vector<BBox3> foot(C->boxes.size());  // stencil footprint per coarse box
  for (auto& b : foot)
    for (int d = 0; d < 3; ++d) {
      b.lo[d] = INT64_MAX;
      b.hi[d] = INT64_MIN;
    }
  // prolongation: per fine box, its buffer-band points and its shell points
  // outside R, assigned to the first coarse box whose interior holds their
  // stencils
  for (size_t fb = 0; fb < F->boxes.size(); ++fb) {
    const sc_box& B = F->boxes[fb];
    const BBox3 bb = box_of(B.lo, B.hi);
    BBoxSet3 todo = ((BBoxSet3::box(bb) - Ts) | (star_shell(bb) - Rs));
    for (size_t cb = 0; cb < C->boxes.size() && !todo.empty(); ++cb) {
      const sc_box& CB = C->boxes[cb];
      const BBoxSet3 part = todo & BBoxSet3::box(safe_fine(CB));
      if (part.empty()) continue;
      todo = todo - part;
      const long long cbase = (long long)(C->off[cb] - CB.lo[0] - CB.lo[1] * C->py[cb] -
                                          CB.lo[2] * C->pz[cb]);
      for (const BBox3& r : part.boxes()) {
        H->prol_rects.push_back({r.lo[0], r.lo[1], r.lo[2], r.hi[0], r.hi[1], r.hi[2]});
        H->n_prol += r.size();
        for (int d = 0; d < 3; ++d) {
          foot[cb].lo[d] = std::min(foot[cb].lo[d], stencil_lo(r.lo[d]));
          foot[cb].hi[d] = std::max(foot[cb].hi[d], stencil_hi(r.hi[d] - 1));
          if (r.hi[d] - r.lo[d] > 1) {
            foot[cb].lo[d] = std::min(foot[cb].lo[d], stencil_lo(r.lo[d] + 1));
            foot[cb].hi[d] = std::max(foot[cb].hi[d], stencil_hi(r.hi[d] - 2));
          }
        }
        // one entry per parity class: points 2 apart along every axis
        for (int k = 0; k < 8; ++k) {
          int64_t s0[3];
          int e[3];
          for (int d = 0; d < 3; ++d) {
            s0[d] = r.lo[d] + ((k >> d) & 1);
            e[d] = s0[d] < r.hi[d] ? (int)((r.hi[d] - s0[d] + 1) / 2) : 0;
          }
          if (!e[0] || !e[1] || !e[2]) continue;
          dev::DProl p{};
          p.dst = elem(F, (int)fb, s0);
          p.dpy = (int)F->py[fb];
          p.dpz = (int)F->pz[fb];
          p.ex = e[0];
          p.ey = e[1];
          p.ez = e[2];
          p.fx0 = (int)s0[0];
          p.fy0 = (int)s0[1];
          p.fz0 = (int)s0[2];
          p.cbase = cbase;
          p.cpy = (int)C->py[cb];
          p.cpz = (int)C->pz[cb];
          H->prol.push_back(p);
          // one chunk per tile of the entry (the tile index in `first`)
          const int ntiles = ((e[0] + dev::kProlTX - 1) / dev::kProlTX) *
                             ((e[1] + dev::kProlTY - 1) / dev::kProlTY) *
                             ((e[2] + dev::kProlTZ - 1) / dev::kProlTZ);
          for (int t = 0; t < ntiles; ++t)
            H->prol_chunks.push_back(dev::DChunk{(int)H->prol.size() - 1, t});
        }
      }
    }
    if (!todo.empty())
      return set_error(SC_EINVAL, "hierarchy: prolongation stencil of fine box " +
                                      std::to_string(fb) +
                                      " lies in no coarse box interior (keep the fine "
                                      "region 3 coarse points away from coarse box faces)");
  }
  for (size_t cb = 0; cb < C->boxes.size(); ++cb) {
    if (foot[cb].lo[0] == INT64_MAX) continue;
    dev::DRect r{};
    r.src = r.dst = elem(C, (int)cb, foot[cb].lo.data());
    r.spy = r.dpy = C->py[cb];
    r.spz = r.dpz = C->pz[cb];
    r.ex = (int)(foot[cb].hi[0] - foot[cb].lo[0]);
    r.ey = (int)(foot[cb].hi[1] - foot[cb].lo[1]);
    r.ez = (int)(foot[cb].hi[2] - foot[cb].lo[2]);
    H->blend.push_back(r);
    add_chunks((int)H->blend.size() - 1, (int64_t)r.ex * r.ey * r.ez, H->blend_chunks,
               dev::kChunk);
  }
  // restriction: coarse points c with 2c in T, per (coarse box, fine box)
  for (size_t cb = 0; cb < C->boxes.size(); ++cb) {
    const sc_box& CB = C->boxes[cb];
    for (size_t fb = 0; fb < F->boxes.size(); ++fb) {
      const sc_box& B = F->boxes[fb];
      const BBoxSet3 part =
          coarsened(Ts & BBoxSet3::box(box_of(B.lo, B.hi)), 2) & BBoxSet3::box(box_of(CB.lo, CB.hi));
      for (const BBox3& r : part.boxes()) {
        dev::DRestr q{};
        q.dst = elem(C, (int)cb, r.lo.data());
        q.dpy = (int)C->py[cb];
        q.dpz = (int)C->pz[cb];
        q.ex = (int)(r.hi[0] - r.lo[0]);
        q.ey = (int)(r.hi[1] - r.lo[1]);
        q.ez = (int)(r.hi[2] - r.lo[2]);
        const int64_t f0[3] = {2 * r.lo[0], 2 * r.lo[1], 2 * r.lo[2]};
        q.src = elem(F, (int)fb, f0);
        q.spy = (int)F->py[fb];
        q.spz = (int)F->pz[fb];
        H->restr.push_back(q);
        H->restr_rects.push_back({r.lo[0], r.lo[1], r.lo[2], r.hi[0], r.hi[1], r.hi[2]});
        const int64_t n = (int64_t)q.ex * q.ey * q.ez;
        add_chunks((int)H->restr.size() - 1, n, H->restr_chunks);
        H->n_restr += n;
      }
    }
  }
  return check_lists(H);
}

// Host check of the device lists before upload: every element an entry
// reads or writes lies in its level's field (fields hold field_size
// elements).  A list built wrong fails here, not on the device.
bool span_in(int64_t e0, int64_t sx, int64_t sy, int64_t sz, int64_t ex, int64_t ey, int64_t ez,
             int64_t n) {
  if (ex <= 0 || ey <= 0 || ez <= 0) return true;
  return e0 >= 0 && e0 + (ex - 1) * sx + (ey - 1) * sy + (ez - 1) * sz < n;
}

int check_lists(const sc_hierarchy* H) {
  const int64_t nc = H->coarse->field_size, nf = H->fine->field_size;
  for (const dev::DProl& p : H->prol) {
    // the fine targets, two apart along each axis
    if (!span_in(p.dst, 2, 2 * (int64_t)p.dpy, 2 * (int64_t)p.dpz, p.ex, p.ey, p.ez, nf))
      return set_error(SC_EINVAL, "internal: a prolongation target lies outside the fine field");
    // the coarse stencil points of the first and the last target
    const int64_t f0[3] = {p.fx0, p.fy0, p.fz0};
    const int64_t f1[3] = {p.fx0 + 2 * (int64_t)(p.ex - 1), p.fy0 + 2 * (int64_t)(p.ey - 1),
                           p.fz0 + 2 * (int64_t)(p.ez - 1)};
    const int64_t lo = p.cbase + stencil_lo(f0[0]) + stencil_lo(f0[1]) * p.cpy +
                       stencil_lo(f0[2]) * p.cpz;
    const int64_t hi = p.cbase + (stencil_hi(f1[0]) - 1) + (stencil_hi(f1[1]) - 1) * p.cpy +
                       (stencil_hi(f1[2]) - 1) * p.cpz;
    if (lo < 0 || hi >= nc)
      return set_error(SC_EINVAL, "internal: a prolongation stencil lies outside the coarse field");
  }
  for (const dev::DRect& r : H->blend)
    if (!span_in(r.src, 1, r.spy, r.spz, r.ex, r.ey, r.ez, nc))
      return set_error(SC_EINVAL, "internal: a coarse footprint lies outside the coarse field");
  for (const dev::DRestr& q : H->restr)
    if (!span_in(q.dst, 1, q.dpy, q.dpz, q.ex, q.ey, q.ez, nc) ||
        !span_in(q.src, 2, 2 * (int64_t)q.spy, 2 * (int64_t)q.spz, q.ex, q.ey, q.ez, nf))
      return set_error(SC_EINVAL, "internal: a restriction entry lies outside its fields");
  return SC_OK;
}

int ensure_uploaded(sc_hierarchy* H) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return set_error(SC_ECUDA, "cudaGetDevice failed");
  if (H->device == cur) return SC_OK;
  if (H->device >= 0) return set_error(SC_EINVAL, "hierarchy was set up on another device");
  int rc;
  if ((rc = upload(&H->d_prol, H->prol)) || (rc = upload(&H->d_prol_chunks, H->prol_chunks)) ||
      (rc = upload(&H->d_blend, H->blend)) || (rc = upload(&H->d_blend_chunks, H->blend_chunks)) ||
      (rc = upload(&H->d_restr, H->restr)) ||
      (rc = upload(&H->d_restr_chunks, H->restr_chunks)))
    return rc;
  H->device = cur;
  return SC_OK;
}

int cuda_check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return SC_OK;
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int write_points(const std::vector<std::array<int64_t, 6>>& rects, int64_t* xyz, int64_t cap,
                 int64_t* n) {
  int64_t k = 0;
  for (const auto& r : rects)
    for (int64_t z = r[2]; z < r[5]; ++z)
      for (int64_t y = r[1]; y < r[4]; ++y)
        for (int64_t x = r[0]; x < r[3]; ++x, ++k)
          if (xyz && k < cap) {
            xyz[3 * k] = x;
            xyz[3 * k + 1] = y;
            xyz[3 * k + 2] = z;
          }
  *n = k;
  return SC_OK;
}

}  // namespace
}  // namespace sc

using namespace sc;

extern "C" {

int sc_hierarchy_create(sc_level* coarse, sc_level* fine, int32_t ratio, int32_t buffer,
                        sc_hierarchy** out) {
  if (!coarse || !fine || !out) return set_error(SC_EINVAL, "NULL argument");
  *out = nullptr;
  if (coarse->partial || fine->partial)
    return set_error(SC_EINVAL, "hierarchy: levels must not be distributed (sc_dist_create)");
  if (ratio != 2) return set_error(SC_EINVAL, "hierarchy: refinement ratio must be 2");
  if (buffer < 4) return set_error(SC_EINVAL, "hierarchy: buffer must be >= 4");
  if (coarse->doms.size() != 1 || fine->doms.size() != 1)
    return set_error(SC_EINVAL, "hierarchy: each level must have exactly one domain");
  const sc_domain& CD = coarse->doms[0];
  const sc_domain& FD = fine->doms[0];
  if (CD.periodic != 7u)
    return set_error(SC_EINVAL, "hierarchy: the coarse domain must be periodic on every axis");
  if (FD.periodic != 0u)
    return set_error(SC_EINVAL, "hierarchy: the fine domain must be periodic on no axis");
  if (!(FD.h == 0.5 * CD.h))
    return set_error(SC_EINVAL, "hierarchy: the fine spacing must be half the coarse spacing");
  sc_hierarchy* H = new sc_hierarchy;
  H->coarse = coarse;
  H->fine = fine;
  H->buffer = buffer;
  H->R = box_of(FD.lo, FD.hi);
  for (int d = 0; d < 3; ++d) {
    H->T.lo[d] = FD.lo[d] + buffer;
    H->T.hi[d] = FD.hi[d] - buffer;
  }
  if (H->T.empty()) {
    delete H;
    return set_error(SC_EINVAL, "hierarchy: the fine domain has no points beyond its buffer");
  }
  const int rc = build_lists(H);
  if (rc) {
    delete H;
    return rc;
  }
  *out = H;
  return SC_OK;
}

void sc_hierarchy_destroy(sc_hierarchy* H) {
  if (!H) return;
  if (H->device >= 0) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != H->device) cudaSetDevice(H->device);
    cudaDeviceSynchronize();
    cudaFree(H->d_prol);
    cudaFree(H->d_prol_chunks);
    cudaFree(H->d_blend);
    cudaFree(H->d_blend_chunks);
    cudaFree(H->d_restr);
    cudaFree(H->d_restr_chunks);
    if (cur != H->device && cur >= 0) cudaSetDevice(cur);
  }
  delete H;
}

int sc_hierarchy_counts(const sc_hierarchy* H, int64_t* n_prolong, int64_t* n_restrict) {
  if (!H || !n_prolong || !n_restrict) return set_error(SC_EINVAL, "NULL argument");
  *n_prolong = H->n_prol;
  *n_restrict = H->n_restr;
  return SC_OK;
}

int sc_hierarchy_prolongation_points(const sc_hierarchy* H, int64_t* xyz, int64_t cap,
                                     int64_t* n) {
  if (!H || !n) return set_error(SC_EINVAL, "NULL argument");
  return write_points(H->prol_rects, xyz, cap, n);
}

int sc_hierarchy_restriction_points(const sc_hierarchy* H, int64_t* xyz, int64_t cap,
                                    int64_t* n) {
  if (!H || !n) return set_error(SC_EINVAL, "NULL argument");
  return write_points(H->restr_rects, xyz, cap, n);
}

namespace {
// Prolongation; emax (or NULL): exponent-bound slots that take the written
// values' exponents in (see sc_hierarchy_step)
int prolongate(sc_hierarchy* H, const double* u0, const double* u1, const double* p0,
               const double* p1, double alpha, double* fu, double* fpi, unsigned* emax,
               void* stream);
int restrict_to(sc_hierarchy* H, const double* fu, const double* fpi, double* cu, double* cpi,
                unsigned* emax, void* stream);
}  // namespace

int sc_hierarchy_prolongate(sc_hierarchy* H, const double* u0, const double* u1, const double* p0,
                            const double* p1, double alpha, double* fu, double* fpi,
                            void* stream) {
  return prolongate(H, u0, u1, p0, p1, alpha, fu, fpi, nullptr, stream);
}

int sc_hierarchy_restrict(sc_hierarchy* H, const double* fu, const double* fpi, double* cu,
                          double* cpi, void* stream) {
  return restrict_to(H, fu, fpi, cu, cpi, nullptr, stream);
}

namespace {
int prolongate(sc_hierarchy* H, const double* u0, const double* u1, const double* p0,
               const double* p1, double alpha, double* fu, double* fpi, unsigned* emax,
               void* stream) {
  if (!H) return set_error(SC_EINVAL, "NULL hierarchy");
  if (!aligned16(u0) || !aligned16(u1) || !aligned16(p0) || !aligned16(p1) || !aligned16(fu) ||
      !aligned16(fpi))
    return set_error(SC_EINVAL, "fields must be 16-byte aligned device pointers");
  int rc = ensure_uploaded(H);
  if (rc) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  const double* du = u0;
  const double* dp = p0;
  if (alpha != 0.0) {
    // the coarse data at t + alpha dt, once per point of the stencils' reach
    double *bu, *bp;
    if ((rc = ensure_device(H->coarse)) || (rc = get_field(H->coarse, "hier.blend.u", &bu)) ||
        (rc = get_field(H->coarse, "hier.blend.pi", &bp)))
      return rc;
    dev::launch_blend(H->d_blend, H->d_blend_chunks, (int)H->blend_chunks.size(), u0, u1, p0,
                      p1, alpha, bu, bp, H->coarse->dev->grid_small, s);
    H->coarse->launches++;
    du = bu;
    dp = bp;
  }
  dev::launch_prolong(H->d_prol, H->d_prol_chunks, (int)H->prol_chunks.size(), du, dp, fu, fpi,
                      emax, s);
  H->fine->launches++;
  return cuda_check("prolongation");
}

int restrict_to(sc_hierarchy* H, const double* fu, const double* fpi, double* cu, double* cpi,
                unsigned* emax, void* stream) {
  if (!H) return set_error(SC_EINVAL, "NULL hierarchy");
  if (!aligned16(fu) || !aligned16(fpi) || !aligned16(cu) || !aligned16(cpi))
    return set_error(SC_EINVAL, "fields must be 16-byte aligned device pointers");
  int rc = ensure_uploaded(H);
  if (rc) return rc;
  dev::launch_restrict(H->d_restr, H->d_restr_chunks, (int)H->restr_chunks.size(), fu, fpi, cu,
                       cpi, emax, (cudaStream_t)stream);
  H->coarse->launches++;
  return cuda_check("restriction");
}
}  // namespace

int sc_hierarchy_step(sc_hierarchy* H, double* cu, double* cpi, const double* cc2, double* fu,
                      double* fpi, const double* fc2, double dt, int32_t nsteps, int32_t mode,
                      void* stream) {
  if (!H) return set_error(SC_EINVAL, "NULL hierarchy");
  if (nsteps < 0 || !(dt >= 0.0)) return set_error(SC_EINVAL, "nsteps < 0 or dt < 0");
  int rc = ensure_uploaded(H);
  if (rc) return rc;
  if ((rc = ensure_device(H->coarse))) return rc;
  double *ou, *op;
  if ((rc = get_field(H->coarse, "hier.old.u", &ou)) ||
      (rc = get_field(H->coarse, "hier.old.pi", &op)))
    return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  const double dtf = 0.5 * dt;
  if ((rc = ensure_device(H->fine))) return rc;
  // Exponent bounds: after its first step in this call a level reuses the
  // bounds its last pass left in the slots of (u, pi) (two stages per pass),
  // raised by the restriction (coarse) or prolongation (fine) that wrote
  // into it since, instead of scanning its fields again
  unsigned* ce = H->coarse->dev->emax;
  unsigned* fe = H->fine->dev->emax;
  for (int n = 0; n < nsteps; ++n) {
    // the coarse level at t where prolongation reads it (the blend with
    // alpha = 0 of a field with itself is that field), then one coarse step
    dev::launch_blend(H->d_blend, H->d_blend_chunks, (int)H->blend_chunks.size(), cu, cu, cpi,
                      cpi, 0.0, ou, op, H->coarse->dev->grid_small, s);
    H->coarse->launches++;
    if ((rc = cuda_check("hierarchy: copy of the coarse level"))) return rc;
    // c2 and dt are fixed within the call: the pre-scaled wave speeds are
    // computed on each level's first step only
    if ((rc = level_steps(H->coarse, cu, cpi, cc2, dt, 1, mode, s, n == 0, n > 0))) return rc;
    // two fine steps of dt/2, boundary data at t and t + dt/2
    for (int k = 0; k < 2; ++k) {
      const bool first = n == 0 && k == 0;
      if ((rc = prolongate(H, ou, cu, op, cpi, 0.5 * k, fu, fpi, first ? nullptr : fe, stream)))
        return rc;
      if ((rc = level_steps(H->fine, fu, fpi, fc2, dtf, 1, mode, s, first, !first))) return rc;
    }
    if ((rc = restrict_to(H, fu, fpi, cu, cpi, ce, stream))) return rc;
  }
  return SC_OK;
}

}  // extern "C"
