// Run-time tuning of the stage kernel's tiles, the GPU counterpart of the
// paper's LoopControl optimiser (arXiv 1308.1343, Sec. 3.2, "Random-Restart
// Hill-Climbing"):
//  * a "loop setup" is (kernel, box-size class, arithmetic, GPU); each is
//    tuned independently, starting from the heuristic default tile;
//  * hill climbing moves to the fastest neighbour (tile_x one step up or
//    down, tile_z doubled or halved) while that improves the time;
//  * at a local optimum it restarts, with small probability, from a random
//    setting, explores that neighbourhood, and keeps whichever is best;
//  * a candidate whose first timed run is slower than abort_factor x the
//    best known time is abandoned at once (cautious exploration);
//  * results are saved to and restored from an on-disk cache (the paper's
//    proposed future work on saving tuned parameters, Sec. 3.3).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <functional>
#include <map>
#include <random>
#include <sstream>
#include <string>
#include <vector>

#include "level.hpp"

namespace sc {
namespace {

struct Cand {
  int tx, tz;
  bool operator<(const Cand& o) const { return tx != o.tx ? tx < o.tx : tz < o.tz; }
  bool operator==(const Cand& o) const { return tx == o.tx && tz == o.tz; }
};

const int kTx[] = {16, 32, 64};

std::string cache_key(const sc_level* L, const SizeClass& c) {
  std::ostringstream k;
  k << L->dev->gpu_name << "|" << L->dev->sms << "|" << L->arith << "|f" << L->fuse
    << (L->fuse == 2 && L->pass_ws ? "w" : "") << "|" << c.ext[0] << "," << c.ext[1] << ","
    << c.ext[2];
  return k.str();
}

// The whole level in one form (two stages per pass with the warp-specialised
// or the one-role kernels, or one stage with either staging): its boxes and
// domains hashed, so that a level's whole-level timings are found again only
// for the same level.
std::string level_key(const sc_level* L) {
  std::ostringstream d;
  for (const auto& B : L->boxes)
    d << B.lo[0] << "," << B.lo[1] << "," << B.lo[2] << ":" << B.hi[0] << "," << B.hi[1] << ","
      << B.hi[2] << "@" << B.domain << ";";
  for (const auto& D : L->doms) d << D.h << "/" << D.periodic << ";";
  std::ostringstream k;
  k << L->dev->gpu_name << "|" << L->dev->sms << "|" << L->arith << "|level"
    << std::hex << std::hash<std::string>{}(d.str()) << "|f" << std::dec << L->fuse;
  if (L->fuse == 2)
    k << (L->pass_ws ? "w" : "o");
  else
    k << "s" << L->staging;
  return k.str();
}

std::map<std::string, std::pair<Cand, double>> read_cache(const char* path) {
  std::map<std::string, std::pair<Cand, double>> m;
  if (!path) return m;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    // key \t tx \t tz \t microseconds
    std::istringstream is(line);
    std::string key;
    Cand c{};
    double us = 0;
    // the file is outside the library's control: an entry is used only if
    // its tile is one the kernels accept (the rules of sc_level_set_tuning)
    if (std::getline(is, key, '\t') && (is >> c.tx >> c.tz >> us) &&
        (c.tx == 16 || c.tx == 32 || c.tx == 64) && c.tz >= 1 && c.tz <= (1 << 20) &&
        std::isfinite(us) && us >= 0.0)
      m[key] = {c, us};
  }
  return m;
}

void write_cache(const char* path, const std::map<std::string, std::pair<Cand, double>>& m) {
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    for (const auto& kv : m)
      f << kv.first << "\t" << kv.second.first.tx << "\t" << kv.second.first.tz << "\t"
        << kv.second.second << "\n";
  }
  std::rename(tmp.c_str(), path);
}

struct Timer {
  sc_level* L;
  cudaStream_t s;
  double* W[6];
  double* c2;
  cudaEvent_t e0, e1;
  dev::DItem* ditems = nullptr;
  size_t cap = 0;

  // Items of the whole level with the current tiles, except class `cls`
  // which gets (tx, tz): the candidate is timed in the launch it will run in
  // (coordinate descent over the classes); cls == kAll gives every class the
  // candidate.  Returns the item count.
  static constexpr int kAll = -2;
  int stage(int cls, const Cand& c) {
    std::vector<dev::DItem> items;
    for (size_t b = 0; b < L->boxes.size(); ++b) {
      const sc_box& B = L->boxes[b];
      const int nx = (int)(B.hi[0] - B.lo[0]), ny = (int)(B.hi[1] - B.lo[1]),
                nz = (int)(B.hi[2] - B.lo[2]);
      const bool mine = cls == kAll || L->box_class[b] == cls;
      const int tx = mine ? c.tx : L->classes[L->box_class[b]].tile.tile_x;
      const int tz = mine ? c.tz : L->classes[L->box_class[b]].tile.tile_z;
      const auto& cuts = L->xcuts;
      const bool cut = cuts.size() == 2 * L->boxes.size();
      append_box_items(items, (int)b, nx, ny, nz, tx, 2 * dev_threads() / tx, tz,
                       cut ? &cuts[2 * b] : nullptr, cut ? &cuts[2 * b + 1] : nullptr);
    }
    order_items(L, items);  // as the level's batched launches run them
    if (items.size() > cap) {
      if (ditems) cudaFree(ditems);
      cap = items.size() * 2;
      if (cudaMalloc(&ditems, cap * sizeof(dev::DItem)) != cudaSuccess) return -1;
    }
    if (cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(dev::DItem),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return -1;
    return (int)items.size();
  }
  static int dev_threads() { return dev::stage_threads(); }

  // The two passes of one step (two stages per pass), on the scratch fields.
  void launch_pairs(int n) {
    DeviceState* D = L->dev;
    const int nd = (int)L->doms.size();
    dev::PairArgs p{};
    p.items = ditems;
    p.nitems = n;
    p.ndom = nd;
    p.boxes = D->boxes;
    p.s0 = p.yu = W[0];
    p.s1 = p.yp = W[1];
    p.q = W[4];
    p.x = W[5];
    p.out_u = W[2];
    p.out_p = W[3];
    p.ly = c2;
    p.coef = D->coef;
    p.emax_in = D->emax;
    p.emax_out = D->emax + 2 * nd;
    p.err = D->err;
    p.xg = D->xg;
    p.xg_ofs = D->xg_ofs;
    launch_pass(L, false, p, s);
    p.s0 = W[2];
    p.s1 = W[3];
    p.x = c2;
    p.out_u = W[0];
    p.out_p = W[1];
    p.ly = nullptr;
    p.emax_in = D->emax + 2 * nd;
    p.emax_out = D->emax;
    launch_pass(L, true, p, s);
  }

  // Median time (microseconds) of what one stencil pass of the level's
  // items costs in the configured form (one stage launch, or the two passes
  // of a step); gives up after the second run if it exceeds `limit`.
  double time(int cls, const Cand& c, double limit) {
    const int n = stage(cls, c);
    if (n <= 0) return 1e30;
    DeviceState* D = L->dev;
    const int nd = (int)L->doms.size();
    dev::FwdArgs a{};
    a.items = ditems;
    a.nitems = n;
    a.ndom = nd;
    a.boxes = D->boxes;
    a.wu_in = W[0];
    a.wp_in = W[1];
    a.yu = W[2];
    a.yp = W[3];
    a.c2 = c2;
    a.q = c2;
    a.qk = 0;
    a.push = D->push;
    a.push_gofs = D->push_gofs;
    a.wu_out = W[2];
    a.wp_out = W[3];
    a.coef = D->coef;
    a.emax_in = D->emax;
    a.emax_out = D->emax + nd;
    a.emax_clear = D->emax + 2 * nd;
    a.err = D->err;
    std::vector<double> ts;
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e0, s);
      if (L->fuse == 2)
        launch_pairs(n);
      else
        dev::launch_fwd_stage(L->arith, false, L->staging, a, D->grid_stage_s[L->staging], s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ts.push_back(ms * 1e3);
      if (r == 1 && ts.back() > limit) return ts.back();  // abort the excursion
    }
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
  }
};

std::vector<Cand> neighbours(const Cand& c, int64_t nz) {
  std::vector<Cand> v;
  const int n = sizeof(kTx) / sizeof(kTx[0]);
  for (int i = 0; i < n; ++i)
    if (kTx[i] == c.tx) {
      if (i > 0) v.push_back(Cand{kTx[i - 1], c.tz});
      if (i + 1 < n) v.push_back(Cand{kTx[i + 1], c.tz});
    }
  if (c.tz > 4) v.push_back(Cand{c.tx, c.tz / 2});
  if (c.tz < nz) v.push_back(Cand{c.tx, c.tz * 2});
  // finer steps: one z-run more or fewer per box column (the runs of a box
  // have near-equal lengths), which moves the item count against the
  // persistent grid's waves
  const int64_t runs = (nz + c.tz - 1) / c.tz;
  for (int64_t r : {runs - 1, runs + 1})
    if (r >= 1 && r <= nz) {
      const int tz = (int)((nz + r - 1) / r);
      if (tz >= 4 && tz != c.tz) v.push_back(Cand{c.tx, tz});
    }
  return v;
}

// Tune the tile of every size class for the level's current form (stages
// per pass): per class, hill climbing with random restarts from the class's
// current tile, or the cached result.  Returns the time (microseconds) of
// one step's stencil launches with the tuned tiles, or a negative value if
// a launch failed.
double tune_form(sc_level* L, Timer& T, std::map<std::string, std::pair<Cand, double>>& cache,
                 std::mt19937_64& rng, double per_class, double abort_factor) {
  cudaStream_t s = T.s;
  std::uniform_real_distribution<double> U(0.0, 1.0);
  // Many size classes (a level of uneven boxes): first one tile for every
  // class not in the cache, hill climbing over the whole level with half of
  // the budget, so that each class starts its own search from it.
  size_t uncached = 0;
  int64_t nzmax = 1;
  std::vector<sc_tile> shared;     // every class's tile after the shared phase
  std::vector<char> refined_here;  // the class is tuned here (not from the cache)
  for (const auto& C : L->classes) {
    if (!cache.count(cache_key(L, C))) ++uncached;
    nzmax = std::max(nzmax, C.ext[2]);
  }
  if (uncached >= 4) {
    std::map<Cand, double> seen;
    auto eval = [&](const Cand& c, double limit) {
      auto it = seen.find(c);
      if (it != seen.end()) return it->second;
      const double t = T.time(Timer::kAll, c, limit);
      seen[c] = t;
      return t;
    };
    Cand best{L->classes[0].tile.tile_x, L->classes[0].tile.tile_z};
    double tbest = eval(best, 1e30);
    const double budget = 0.5 * per_class * (double)L->classes.size();
    cudaEvent_t w0, w1;
    cudaEventCreate(&w0);
    cudaEventCreate(&w1);
    cudaEventRecord(w0, s);
    for (double spent = 0; spent < budget;) {
      Cand nb = best;
      double tn = tbest;
      for (const Cand& c : neighbours(best, nzmax)) {
        const double t = eval(c, abort_factor * tbest);
        if (t < tn) {
          tn = t;
          nb = c;
        }
      }
      if (nb == best) break;  // local optimum of the shared tile
      best = nb;
      tbest = tn;
      cudaEventRecord(w1, s);
      cudaEventSynchronize(w1);
      float ms = 0;
      cudaEventElapsedTime(&ms, w0, w1);
      spent = ms;
    }
    cudaEventDestroy(w0);
    cudaEventDestroy(w1);
    for (auto& C : L->classes)
      if (!cache.count(cache_key(L, C))) {
        C.tile.tile_x = best.tx;
        C.tile.tile_y = 2 * dev::stage_threads() / best.tx;
        C.tile.tile_z = (int)std::min<int64_t>(best.tz, C.ext[2]);
      }
    per_class *= 0.5;
    shared.reserve(L->classes.size());
    for (const auto& C : L->classes) {
      shared.push_back(C.tile);
      refined_here.push_back(!cache.count(cache_key(L, C)));
    }
  }
  for (size_t ci = 0; ci < L->classes.size(); ++ci) {
    SizeClass& C = L->classes[ci];
    const std::string key = cache_key(L, C);
    auto hit = cache.find(key);
    if (hit != cache.end()) {
      C.tile.tile_x = hit->second.first.tx;
      C.tile.tile_y = 2 * dev::stage_threads() / hit->second.first.tx;
      C.tile.tile_z = hit->second.first.tz;
      C.fixed = true;
      continue;
    }
    std::map<Cand, double> seen;
    auto eval = [&](const Cand& c, double limit) {
      auto it = seen.find(c);
      if (it != seen.end()) return it->second;
      const double t = T.time((int)ci, c, limit);
      seen[c] = t;
      return t;
    };
    Cand best{C.tile.tile_x, C.tile.tile_z};
    double tbest = eval(best, 1e30);
    Cand cur = best;
    double tcur = tbest;
    cudaEvent_t w0, w1;
    cudaEventCreate(&w0);
    cudaEventCreate(&w1);
    cudaEventRecord(w0, s);
    double spent = 0;
    while (spent < per_class) {
      // hill climbing: move to the best improving neighbour
      Cand nb = cur;
      double tn = tcur;
      for (const Cand& c : neighbours(cur, C.ext[2])) {
        const double t = eval(c, abort_factor * tbest);
        if (t < tn) {
          tn = t;
          nb = c;
        }
      }
      if (nb == cur) {
        // local optimum: restart from a random setting with small probability
        if (U(rng) < 0.25) {
          const int ntx = sizeof(kTx) / sizeof(kTx[0]);
          Cand r{kTx[rng() % ntx], 4 << (rng() % 6)};
          const double t = eval(r, abort_factor * tbest);
          cur = r;
          tcur = t;
        } else if (seen.size() >= 24) {
          break;
        } else {
          cur = best;
          tcur = tbest;
          if (U(rng) < 0.5) break;
        }
      } else {
        cur = nb;
        tcur = tn;
      }
      if (tcur < tbest) {
        tbest = tcur;
        best = cur;
      }
      cudaEventRecord(w1, s);
      cudaEventSynchronize(w1);
      float ms = 0;
      cudaEventElapsedTime(&ms, w0, w1);
      spent = ms;
    }
    cudaEventDestroy(w0);
    cudaEventDestroy(w1);
    C.tile.tile_x = best.tx;
    C.tile.tile_y = 2 * dev::stage_threads() / best.tx;
    C.tile.tile_z = best.tz;
    C.fixed = true;
    cache[key] = {best, tbest};
  }
  // the whole level with every class at its tuned tile.  When every class's
  // tile came from the cache, the whole level's time in this form is taken
  // from the cache too, so that a warm cache reproduces the choice between
  // forms without timing again (a timing taken under a profiler, with its
  // per-launch overhead, could otherwise flip it)
  const bool all_cached = uncached == 0;
  auto level_time = [&]() {
    const std::string key = level_key(L);
    auto it = cache.find(key);
    if (all_cached && it != cache.end()) return it->second.second;
    const double tl = T.time(-1, Cand{0, 0}, 1e30);
    if (tl < 1e30)
      cache[key] = {Cand{L->classes[0].tile.tile_x, L->classes[0].tile.tile_z}, tl};
    return tl;
  };
  double t = level_time();
  if (t >= 1e30) return -1.0;
  // With many classes each class holds a small share of the level's time, and
  // one class's candidates differ by less than the timing noise of the whole
  // level: the per-class refinement may end slower than the shared tile it
  // started from (measured on the uneven 64-box level: 31.5-32.6 against
  // 32.7 G updates/s).  Keep whichever of the two assignments is faster.
  if (!shared.empty()) {
    std::vector<sc_tile> refined;
    for (const auto& C : L->classes) refined.push_back(C.tile);
    for (size_t i = 0; i < L->classes.size(); ++i)
      if (refined_here[i]) L->classes[i].tile = shared[i];
    const double t0 = T.time(-1, Cand{0, 0}, 1e30);
    if (t0 < t) {
      t = t0;
      cache[level_key(L)].second = t0;
      for (size_t i = 0; i < L->classes.size(); ++i) {
        const SizeClass& C = L->classes[i];
        auto it = cache.find(cache_key(L, C));
        if (refined_here[i] && it != cache.end())
          it->second.first = Cand{C.tile.tile_x, C.tile.tile_z};
      }
    } else {
      for (size_t i = 0; i < L->classes.size(); ++i) L->classes[i].tile = refined[i];
    }
  }
  // one stage per pass: the staging of the raw column and halo values too
  // (registers or cp.async), for the whole level with the tuned tiles
  if (L->fuse == 1 && !L->staging_fixed) {
    const int s0 = L->staging;
    L->staging = 1 - s0;
    const double t1 = level_time();
    if (t1 < t)
      t = t1;
    else
      L->staging = s0;
  }
  return L->fuse == 2 ? t : 4.0 * t;
}

// The two-stage form: unless the caller fixed the pass kernels, tune the
// tiles of the warp-specialised and of the one-role kernels and keep the
// faster kernel with its tiles (another choice between sets of loop kernels).
double tune_two_stage(sc_level* L, Timer& T,
                      std::map<std::string, std::pair<Cand, double>>& cache,
                      std::mt19937_64& rng, double per_class, double abort_factor) {
  if (L->pass_fixed) return tune_form(L, T, cache, rng, per_class, abort_factor);
  std::vector<sc_tile> start;
  for (const auto& c : L->classes) start.push_back(c.tile);
  L->pass_ws = 1;
  const double tw = tune_form(L, T, cache, rng, per_class, abort_factor);
  std::vector<sc_tile> tiles_ws;
  for (const auto& c : L->classes) tiles_ws.push_back(c.tile);
  for (size_t i = 0; i < L->classes.size(); ++i) L->classes[i].tile = start[i];
  L->pass_ws = 0;
  const double to = tune_form(L, T, cache, rng, per_class, abort_factor);
  if (tw < 0 || to < 0) return -1.0;
  // the one-role tiles stay with the classes for the adjoint's pass kernels
  for (auto& c : L->classes) {
    c.tile_one = c.tile;
    c.has_one = true;
  }
  if (tw <= to) {
    L->pass_ws = 1;
    for (size_t i = 0; i < L->classes.size(); ++i) L->classes[i].tile = tiles_ws[i];
    return tw;
  }
  return to;
}

}  // namespace
}  // namespace sc

using namespace sc;

extern "C" int sc_level_autotune(sc_level* L, int32_t seed, double budget_ms,
                                 double abort_factor, const char* cache_path, void* stream) {
  if (!L) return set_error(SC_EINVAL, "NULL level");
  if (!(abort_factor > 1.0)) return set_error(SC_EINVAL, "abort_factor must be > 1");
  int rc = ensure_device(L);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  Timer T{L, s};
  if ((rc = scratch4(L, T.W)) || (rc = get_field(L, "tune.c2", &T.c2))) return rc;
  const double dt0 = 0.0;
  if ((rc = set_coef(L, &dt0, 1, s))) return rc;
  cudaEventCreate(&T.e0);
  cudaEventCreate(&T.e1);
  auto cache = read_cache(cache_path);
  std::mt19937_64 rng((uint64_t)seed);
  // Unless the caller fixed the form, both are tuned and the faster kept:
  // choosing between sets of loop kernels (one or two RK4 stages per pass)
  // with the same optimiser, as the paper proposes for fission and fusion.
  // tunings: the one-stage form, and the two-stage form with each of its
  // pass kernels
  const int nforms = (L->fuse_fixed && L->fuse == 1 ? 1 : 0) +
                     (L->fuse_fixed && L->fuse == 2 ? (L->pass_fixed ? 1 : 2) : 0) +
                     (L->fuse_fixed ? 0 : (L->pass_fixed ? 2 : 3));
  const double per_class = budget_ms / (nforms * std::max<size_t>(1, L->classes.size()));
  bool ok = true;
  if (L->fuse_fixed) {
    ok = (L->fuse == 2 ? tune_two_stage(L, T, cache, rng, per_class, abort_factor)
                       : tune_form(L, T, cache, rng, per_class, abort_factor)) >= 0;
  } else {
    std::vector<sc_tile> start;
    for (const auto& c : L->classes) start.push_back(c.tile);
    L->fuse = 1;
    const double t1 = tune_form(L, T, cache, rng, per_class, abort_factor);
    std::vector<sc_tile> tiles1;
    for (const auto& c : L->classes) tiles1.push_back(c.tile);
    for (size_t i = 0; i < L->classes.size(); ++i) L->classes[i].tile = start[i];
    L->fuse = 2;
    const double t2 = tune_two_stage(L, T, cache, rng, per_class, abort_factor);
    ok = t1 >= 0 && t2 >= 0;
    if (ok && t1 < t2) {
      L->fuse = 1;
      for (size_t i = 0; i < L->classes.size(); ++i) L->classes[i].tile = tiles1[i];
    }
  }
  if (T.ditems) cudaFree(T.ditems);
  cudaEventDestroy(T.e0);
  cudaEventDestroy(T.e1);
  write_cache(cache_path, cache);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SC_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
  if (!ok) return set_error(SC_ECUDA, "autotune: a timed launch failed");
  return upload_items(L);
}
