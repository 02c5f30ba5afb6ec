// Bounding-box-set algebra stored as discrete derivatives (arXiv 1308.1343,
// Sec. 2).
//
// A D-dimensional set R of integer grid points is represented by its discrete
// derivative along the last axis, d = D-1:
//     (d_d R)(p) = R(p) xor R(p - e_d)
// i.e. an ordered map from each position n along axis d where the
// (D-1)-dimensional cross-section of R changes to that change
// (cross-section(n) xor cross-section(n-1)), itself a (D-1)-dimensional set
// stored the same way; the recursion ends at D = 0, a single boolean
// (Sec. 2.3, dimensional recursion).  The representation is canonical:
// empty changes are never stored, so two sets are equal iff their maps are.
//
// Binary operations T = R (op) S use the sweep of Sec. 2.3 (Fig.
// "bboxset-traverse"): walk the union of the stored positions of R and S in
// increasing order, update the current cross-sections r, s by xor with the
// stored change, recompute t = r (op) s one dimension down, and store
// t xor t_previous when it is not empty.  The symmetric difference needs no
// sweep: it is the xor of the stored derivatives (Eq. "xor").
#pragma once

#include <algorithm>
#include <array>
#include <cstdint>
#include <map>
#include <vector>

namespace sc {

enum class SetOp { Union, Intersection, Difference, Xor };

inline bool apply_op(SetOp op, bool a, bool b) {
  switch (op) {
    case SetOp::Union: return a || b;
    case SetOp::Intersection: return a && b;
    case SetOp::Difference: return a && !b;
    case SetOp::Xor: return a != b;
  }
  return false;
}

template <int D>
struct Box {
  std::array<int64_t, D> lo{}, hi{};
  bool empty() const {
    for (int d = 0; d < D; ++d)
      if (lo[d] >= hi[d]) return true;
    return false;
  }
  int64_t size() const {
    if (empty()) return 0;
    int64_t n = 1;
    for (int d = 0; d < D; ++d) n *= hi[d] - lo[d];
    return n;
  }
  bool operator<(const Box& o) const {
    for (int d = D - 1; d >= 0; --d) {
      if (lo[d] != o.lo[d]) return lo[d] < o.lo[d];
      if (hi[d] != o.hi[d]) return hi[d] < o.hi[d];
    }
    return false;
  }
  bool operator==(const Box& o) const { return lo == o.lo && hi == o.hi; }
};

template <int D>
struct BBoxSet;

// D = 0: a single point that is either in the set or not.
template <>
struct BBoxSet<0> {
  bool v = false;

  static BBoxSet box(const int64_t*, const int64_t*) { return BBoxSet{true}; }
  bool empty() const { return !v; }
  bool operator==(const BBoxSet& o) const { return v == o.v; }
  void xor_with(const BBoxSet& o) { v = (v != o.v); }
  static BBoxSet binop(const BBoxSet& r, const BBoxSet& s, SetOp op) {
    return BBoxSet{apply_op(op, r.v, s.v)};
  }
  BBoxSet shifted(const int64_t*) const { return *this; }
  int64_t size() const { return v ? 1 : 0; }
  void boxes(std::vector<Box<0>>& out) const {
    if (v) out.push_back(Box<0>{});
  }
  void derivative_points(std::vector<std::array<int64_t, 0>>& out) const {
    if (v) out.push_back({});
  }
};

template <int D>
struct BBoxSet {
  static_assert(D >= 1, "dimension");
  using Sub = BBoxSet<D - 1>;
  // position along axis D-1 -> change of the (D-1)-dimensional cross-section
  std::map<int64_t, Sub> m;

  bool empty() const { return m.empty(); }
  bool operator==(const BBoxSet& o) const { return m == o.m; }
  bool operator!=(const BBoxSet& o) const { return !(m == o.m); }

  // The set of all points of [lo, hi): its cross-section switches on at
  // lo[D-1] and off at hi[D-1].
  static BBoxSet box(const int64_t* lo, const int64_t* hi) {
    BBoxSet r;
    for (int d = 0; d < D; ++d)
      if (lo[d] >= hi[d]) return r;
    Sub c = Sub::box(lo, hi);
    r.m.emplace(lo[D - 1], c);
    r.m.emplace(hi[D - 1], c);
    return r;
  }
  static BBoxSet box(const Box<D>& b) { return box(b.lo.data(), b.hi.data()); }

  // Symmetric difference directly on the stored derivatives (Eq. "xor").
  void xor_with(const BBoxSet& o) {
    for (const auto& kv : o.m) {
      auto it = m.find(kv.first);
      if (it == m.end()) {
        m.emplace(kv.first, kv.second);
      } else {
        it->second.xor_with(kv.second);
        if (it->second.empty()) m.erase(it);
      }
    }
  }

  // The sweep of Sec. 2.3 for an arbitrary pointwise set operation.
  static BBoxSet binop(const BBoxSet& R, const BBoxSet& S, SetOp op) {
    if (op == SetOp::Xor) {
      BBoxSet t = R;
      t.xor_with(S);
      return t;
    }
    BBoxSet T;
    Sub r, s, t;
    auto ir = R.m.begin(), is = S.m.begin();
    while (ir != R.m.end() || is != S.m.end()) {
      // next position at which either stored derivative has an element
      int64_t n;
      if (is == S.m.end() || (ir != R.m.end() && ir->first < is->first))
        n = ir->first;
      else
        n = is->first;
      if (ir != R.m.end() && ir->first == n) { r.xor_with(ir->second); ++ir; }
      if (is != S.m.end() && is->first == n) { s.xor_with(is->second); ++is; }
      Sub t_new = Sub::binop(r, s, op);
      Sub change = t_new;
      change.xor_with(t);
      if (!change.empty()) T.m.emplace_hint(T.m.end(), n, std::move(change));
      t = std::move(t_new);
    }
    return T;
  }

  BBoxSet operator|(const BBoxSet& o) const { return binop(*this, o, SetOp::Union); }
  BBoxSet operator&(const BBoxSet& o) const { return binop(*this, o, SetOp::Intersection); }
  BBoxSet operator-(const BBoxSet& o) const { return binop(*this, o, SetOp::Difference); }
  BBoxSet operator^(const BBoxSet& o) const { return binop(*this, o, SetOp::Xor); }

  // shift(R, v): every stored position moves by v (Sec. 2, `shift`).
  BBoxSet shifted(const int64_t* v) const {
    BBoxSet r;
    for (const auto& kv : m)
      r.m.emplace_hint(r.m.end(), kv.first + v[D - 1], kv.second.shifted(v));
    return r;
  }

  // expand: grow by lo_by[d] below and hi_by[d] above along every axis, the
  // union of the shifts of R by all vectors in the box [-lo_by, hi_by].
  BBoxSet expanded(const int64_t* lo_by, const int64_t* hi_by) const {
    BBoxSet r = *this;
    for (int d = 0; d < D; ++d) {
      BBoxSet acc = r;
      for (int64_t k = -lo_by[d]; k <= hi_by[d]; ++k) {
        if (k == 0) continue;
        int64_t v[D > 0 ? D : 1] = {};
        v[d] = k;
        acc = acc | r.shifted(v);
      }
      r = std::move(acc);
    }
    return r;
  }

  int64_t size() const {
    int64_t n = 0;
    Sub r;
    auto it = m.begin();
    while (it != m.end()) {
      r.xor_with(it->second);
      auto nx = std::next(it);
      if (nx != m.end()) n += r.size() * (nx->first - it->first);
      it = nx;
    }
    return n;
  }

  // Normalized box list: sweep along axis D-1; each box of the current
  // cross-section's own normalized list stays open while the cross-section
  // keeps it, and is emitted when it disappears.  Disjoint, deterministic.
  void boxes(std::vector<Box<D>>& out) const {
    std::map<Box<D - 1>, int64_t> open;  // sub-box -> start position
    Sub r;
    for (const auto& kv : m) {
      const int64_t n = kv.first;
      r.xor_with(kv.second);
      std::vector<Box<D - 1>> cur;
      r.boxes(cur);
      std::sort(cur.begin(), cur.end());
      std::map<Box<D - 1>, int64_t> next;
      for (const auto& b : cur) {
        auto it = open.find(b);
        next.emplace(b, it == open.end() ? n : it->second);
      }
      for (const auto& kv2 : open) {
        if (next.find(kv2.first) == next.end()) {
          Box<D> B;
          for (int d = 0; d < D - 1; ++d) {
            B.lo[d] = kv2.first.lo[d];
            B.hi[d] = kv2.first.hi[d];
          }
          B.lo[D - 1] = kv2.second;
          B.hi[D - 1] = n;
          out.push_back(B);
        }
      }
      open.swap(next);
    }
  }

  std::vector<Box<D>> boxes() const {
    std::vector<Box<D>> v;
    boxes(v);
    return v;
  }

  // Points of the full derivative d_0 ... d_{D-1} R, sorted with the last
  // axis outermost.
  void derivative_points(std::vector<std::array<int64_t, D>>& out) const {
    for (const auto& kv : m) {
      std::vector<std::array<int64_t, D - 1>> sub;
      kv.second.derivative_points(sub);
      for (const auto& p : sub) {
        std::array<int64_t, D> q;
        for (int d = 0; d < D - 1; ++d) q[d] = p[d];
        q[D - 1] = kv.first;
        out.push_back(q);
      }
    }
  }
};

using BBox3 = Box<3>;
using BBoxSet3 = BBoxSet<3>;

inline BBoxSet3 set_of(const std::vector<BBox3>& bs) {
  BBoxSet3 s;
  for (const auto& b : bs) s = s | BBoxSet3::box(b);
  return s;
}

// Spacing change (Sec. 2 lists it among the bboxset operations): the
// points c of the grid with r times the spacing whose position coincides
// with a point of S, {c : r c in S} (vertex-centred grids sharing the
// origin).  A preimage commutes with union, so the normalized boxes can be
// mapped one by one: [lo, hi) -> [ceil(lo / r), ceil(hi / r)).
inline int64_t ceil_div(int64_t a, int64_t r) { return a >= 0 ? (a + r - 1) / r : -((-a) / r); }

inline BBoxSet3 coarsened(const BBoxSet3& S, int64_t r) {
  BBoxSet3 out;
  for (const BBox3& b : S.boxes()) {
    BBox3 c;
    for (int d = 0; d < 3; ++d) {
      c.lo[d] = ceil_div(b.lo[d], r);
      c.hi[d] = ceil_div(b.hi[d], r);
    }
    if (!c.empty()) out = out | BBoxSet3::box(c);
  }
  return out;
}

}  // namespace sc
