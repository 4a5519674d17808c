// Auto-tuning of all kernels' launch and tiling parameters together: the
// genetic algorithm of Sec. 3.2 (initialisation, tournament selection,
// crossover, mutation, replacement of the fitter halves), pure random search
// and exhaustive search (Sec. 4), over a discrete space of genes grouped by
// kernel.  Fitness is the measured run time of the whole search path (Sec. 3.2:
// the run time of the whole pipeline), lower is better; a configuration that
// fails or exceeds the time limit scores +inf (the penalty of Sec. 4).
//
// The engine (sps_optimize) is host code driven by caller callbacks, so it
// runs and is tested without a GPU; sps_tune drives it with the plan's own
// gene space and live timings of the plan's kernels.
//
// Random numbers: SplitMix64 (Steele, Lea & Flood 2014), counter-based:
// output n = mix(seed + n * 0x9E3779B97F4A7C15).  Integers in [0, n) take the
// top 53 bits as a fraction times n; probabilities compare the same fraction.
// The order of draws is part of the algorithm's definition:
//   init:      per individual, one draw per gene, redrawn until valid;
//   selection: per tournament, a partial Fisher-Yates shuffle of N_pop
//              indices for N_pool draws; the fittest (then lowest index) wins;
//   pairing:   Fisher-Yates shuffle of the selected list (from the top);
//   crossover: per pair and kernel, one draw against p_cross; then per gene a
//              coin (> 0.5 swaps) for uniform crossover, or one cut in
//              [0, n_genes_of_kernel) for one-point crossover;
//   mutation:  per offspring and kernel, one draw against p_mut; then the gene
//              index and a new value among the other values;
//   renewal:   per offspring that repeats an evaluated individual or an
//              earlier offspring, per try: the kernel, the gene index and a new
//              value among the other values.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <limits>
#include <map>
#include <numeric>
#include <vector>

#include "sps_internal.h"

namespace sps {
namespace {

class SplitMix64 {
 public:
  explicit SplitMix64(uint64_t seed) : s_(seed) {}
  uint64_t next() {
    s_ += 0x9E3779B97F4A7C15ull;
    uint64_t z = s_;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  int32_t below(int64_t n) {
    const unsigned __int128 f = (unsigned __int128)(next() >> 11) * (uint64_t)n;
    return (int32_t)(f >> 53);
  }
  double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }

 private:
  uint64_t s_;
};

typedef std::vector<int32_t> Point;
const double kInf = std::numeric_limits<double>::infinity();

struct Problem {
  std::vector<int32_t> n_values;
  std::vector<std::vector<int32_t>> kernels;  // gene indices per kernel, in order
  std::function<bool(const Point&)> valid;
  std::function<double(const Point&)> fitness;
  std::function<void(int64_t, const Point&, double)> trace;
  std::function<void(int32_t, int64_t, double, const Point&)> progress;
  std::map<Point, double> known;  // logged evaluations served instead of measuring (resume)
};

class Evaluator {
 public:
  Evaluator(const Problem& pr, int64_t budget) : pr_(pr), budget_(budget) {}
  double operator()(const Point& p) {
    auto it = cache_.find(p);
    if (it != cache_.end()) return it->second;
    if (budget_ >= 0 && count_ >= budget_) return kInf;
    const auto k = pr_.known.find(p);
    double f = k != pr_.known.end() ? k->second : pr_.fitness(p);
    if (std::isnan(f)) f = kInf;
    cache_.emplace(p, f);
    if (pr_.trace) pr_.trace(count_, p, f);
    count_++;
    if (f < best_) {  // ties keep the earlier point
      best_ = f;
      best_point_ = p;
    }
    return f;
  }
  bool seen(const Point& p) const { return cache_.count(p) != 0; }
  int64_t count() const { return count_; }
  double best() const { return best_; }
  const Point& best_point() const { return best_point_; }

 private:
  const Problem& pr_;
  int64_t budget_;
  int64_t count_ = 0;
  double best_ = kInf;
  Point best_point_;
  std::map<Point, double> cache_;
};

bool random_valid(const Problem& pr, SplitMix64& rng, Point* out) {
  Point p(pr.n_values.size());
  for (int tries = 0; tries < 1000; tries++) {
    for (size_t g = 0; g < p.size(); g++) p[g] = rng.below(pr.n_values[g]);
    if (pr.valid(p)) {
      *out = p;
      return true;
    }
  }
  return false;
}

// One gene to a different value drawn uniformly; if that breaks a boundary
// condition the next values in cyclic order are tried, and the old value is
// kept if none is valid.
void mutate_gene(const Problem& pr, Point& c, int32_t g, SplitMix64& rng) {
  const int32_t nv = pr.n_values[g];
  if (nv < 2) return;
  const int32_t old = c[g];
  int32_t v = rng.below(nv - 1);
  if (v >= old) v++;
  int32_t chosen = old;
  for (int32_t s = 0; s < nv; s++) {
    const int32_t cand = (v + s) % nv;
    if (cand == old) continue;
    c[g] = cand;
    if (pr.valid(c)) {
      chosen = cand;
      break;
    }
  }
  c[g] = chosen;
}

sps_status run_genetic(const Problem& pr, const sps_search_desc& d, Point* best, sps_search_result* res) {
  const int32_t n = d.population;
  if (n < 2 || n % 2) return fail(SPS_ERR_INVALID_ARG, "population must be even and >= 2");
  if (!(d.pool_fraction > 0.0)) return fail(SPS_ERR_INVALID_ARG, "pool_fraction must be > 0");
  if (d.renew < 0) return fail(SPS_ERR_INVALID_ARG, "renew must be >= 0");
  SplitMix64 rng(d.seed);
  Evaluator ev(pr, d.max_evaluations);
  const int32_t n_pool = std::min(n, std::max<int32_t>(2, (int32_t)std::floor(d.pool_fraction * n + 0.5)));

  std::vector<Point> pop(n);
  std::vector<double> fit(n);
  for (int32_t j = 0; j < n; j++)
    if (!random_valid(pr, rng, &pop[j])) return fail(SPS_ERR_INVALID_ARG, "no valid individual found");
  for (int32_t j = 0; j < n; j++) fit[j] = ev(pop[j]);
  if (pr.progress) pr.progress(0, ev.count(), ev.best(), ev.best_point());

  int32_t gen = 0;
  std::vector<int32_t> idx(n);
  while (ev.count() < d.max_evaluations && gen < d.max_generations) {
    gen++;
    // selection: N_pop tournaments
    std::vector<Point> sel(n);
    for (int32_t j = 0; j < n; j++) {
      std::iota(idx.begin(), idx.end(), 0);
      for (int32_t q = 0; q < n_pool; q++) std::swap(idx[q], idx[q + rng.below(n - q)]);
      int32_t win = idx[0];
      for (int32_t q = 1; q < n_pool; q++) {
        const int32_t c = idx[q];
        if (fit[c] < fit[win] || (fit[c] == fit[win] && c < win)) win = c;
      }
      sel[j] = pop[win];
    }
    // pairing
    for (int32_t q = n - 1; q > 0; q--) std::swap(sel[q], sel[rng.below(q + 1)]);
    for (int32_t q = 0; q < n; q += 2)
      if (sel[q] == sel[q + 1])
        for (int32_t r = q + 2; r < n; r++)
          if (sel[r] != sel[q]) {
            std::swap(sel[q + 1], sel[r]);
            break;
          }
    // crossover
    std::vector<Point> off = sel;
    for (int32_t q = 0; q < n; q += 2) {
      Point& a = off[q];
      Point& b = off[q + 1];
      for (const auto& genes : pr.kernels) {
        if (!(rng.unit() < d.p_cross)) continue;
        if (d.crossover == SPS_CROSS_UNIFORM) {
          for (int32_t g : genes) {
            if (rng.unit() > 0.5) {
              std::swap(a[g], b[g]);
              if (!(pr.valid(a) && pr.valid(b))) std::swap(a[g], b[g]);
            }
          }
        } else {
          const int32_t cut = rng.below((int64_t)genes.size());
          for (size_t k = cut; k < genes.size(); k++) std::swap(a[genes[k]], b[genes[k]]);
          if (!(pr.valid(a) && pr.valid(b)))
            for (size_t k = cut; k < genes.size(); k++) std::swap(a[genes[k]], b[genes[k]]);
        }
      }
    }
    // mutation
    for (Point& c : off) {
      for (const auto& genes : pr.kernels) {
        if (!(rng.unit() < d.p_mut)) continue;
        mutate_gene(pr, c, genes[rng.below((int64_t)genes.size())], rng);
      }
    }
    // renewal: an offspring that repeats an evaluated individual or an earlier
    // offspring of this generation mutates again (a kernel, then one of its
    // genes), up to `renew` times
    for (int32_t j = 0; j < n; j++) {
      Point& c = off[j];
      for (int32_t tries = 0; tries < d.renew; tries++) {
        bool repeat = ev.seen(c);
        for (int32_t q = 0; q < j && !repeat; q++) repeat = off[q] == c;
        if (!repeat) break;
        const auto& genes = pr.kernels[rng.below((int64_t)pr.kernels.size())];
        mutate_gene(pr, c, genes[rng.below((int64_t)genes.size())], rng);
      }
    }
    std::vector<double> off_fit(n);
    for (int32_t j = 0; j < n; j++) off_fit[j] = ev(off[j]);
    // replacement: fitter half of parents, then fitter half of offspring; an
    // offspring left unevaluated because the budget ran out takes no place and
    // the next-fittest parents fill the population instead
    auto ranked = [&](const std::vector<double>& f, std::vector<int32_t> r, int32_t keep) {
      std::stable_sort(r.begin(), r.end(), [&](int32_t x, int32_t y) { return f[x] < f[y]; });
      r.resize(std::min<size_t>(r.size(), (size_t)keep));
      return r;
    };
    std::vector<int32_t> all(n), evaluated;
    std::iota(all.begin(), all.end(), 0);
    for (int32_t j = 0; j < n; j++)
      if (ev.seen(off[j])) evaluated.push_back(j);
    const std::vector<int32_t> ro = ranked(off_fit, evaluated, n / 2);
    const std::vector<int32_t> rp = ranked(fit, all, n - (int32_t)ro.size());
    std::vector<Point> np;
    std::vector<double> nf;
    for (int32_t j : rp) { np.push_back(pop[j]); nf.push_back(fit[j]); }
    for (int32_t j : ro) { np.push_back(off[j]); nf.push_back(off_fit[j]); }
    pop.swap(np);
    fit.swap(nf);
    if (pr.progress) pr.progress(gen, ev.count(), ev.best(), ev.best_point());
  }
  if (d.final_population)
    for (int32_t j = 0; j < n; j++)
      std::copy(pop[j].begin(), pop[j].end(), d.final_population + (size_t)j * pop[j].size());
  *best = ev.best_point();
  res->best_fitness = ev.best();
  res->evaluations = ev.count();
  res->generations = gen;
  return SPS_OK;
}

sps_status run_random(const Problem& pr, const sps_search_desc& d, Point* best, sps_search_result* res) {
  SplitMix64 rng(d.seed);
  Evaluator ev(pr, d.max_evaluations);
  int64_t draws = 0;
  const int64_t limit = 100 * std::max<int64_t>(1, d.max_evaluations);
  Point p;
  std::vector<Point> drawn;  // distinct individuals in evaluation order
  while (ev.count() < d.max_evaluations && draws < limit) {
    if (!random_valid(pr, rng, &p)) return fail(SPS_ERR_INVALID_ARG, "no valid individual found");
    draws++;
    if (ev.seen(p)) continue;
    ev(p);
    drawn.push_back(p);
  }
  if (d.final_population && d.population > 0) {
    const size_t ng = pr.n_values.size(), np_ = (size_t)d.population;
    const size_t first = drawn.size() > np_ ? drawn.size() - np_ : 0;
    for (size_t j = 0; j < np_; j++) {
      int32_t* row = d.final_population + j * ng;
      if (first + j < drawn.size())
        std::copy(drawn[first + j].begin(), drawn[first + j].end(), row);
      else
        std::fill(row, row + ng, -1);
    }
  }
  if (pr.progress) pr.progress(0, ev.count(), ev.best(), ev.best_point());
  *best = ev.best_point();
  res->best_fitness = ev.best();
  res->evaluations = ev.count();
  res->generations = 0;
  return SPS_OK;
}

sps_status run_exhaustive(const Problem& pr, Point* best, sps_search_result* res) {
  Evaluator ev(pr, -1);
  Point p(pr.n_values.size(), 0);
  for (;;) {
    if (pr.valid(p)) ev(p);
    int32_t g = (int32_t)p.size() - 1;
    for (; g >= 0; g--) {
      if (++p[g] < pr.n_values[g]) break;
      p[g] = 0;
    }
    if (g < 0) break;
  }
  if (pr.progress) pr.progress(0, ev.count(), ev.best(), ev.best_point());
  *best = ev.best_point();
  res->best_fitness = ev.best();
  res->evaluations = ev.count();
  res->generations = 0;
  return SPS_OK;
}

sps_status run_problem(Problem& pr, const sps_search_desc* d, int32_t* best_point, sps_search_result* res) {
  if (!d || !best_point || !res) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (d->n_known < 0 || (d->n_known > 0 && (!d->known_points || !d->known_fitness)))
    return fail(SPS_ERR_INVALID_ARG, "known evaluations: n_known < 0 or null arrays");
  const size_t n_genes = pr.n_values.size();
  for (int64_t k = 0; k < d->n_known; k++) {
    Point p(d->known_points + k * n_genes, d->known_points + (k + 1) * n_genes);
    for (size_t g = 0; g < n_genes; g++)
      if (p[g] < 0 || p[g] >= pr.n_values[g]) return fail(SPS_ERR_INVALID_ARG, "known point out of the space");
    pr.known.emplace(std::move(p), d->known_fitness[k]);
  }
  Point best;
  sps_status s;
  switch (d->algorithm) {
    case SPS_TUNE_GA: s = run_genetic(pr, *d, &best, res); break;
    case SPS_TUNE_RANDOM: s = run_random(pr, *d, &best, res); break;
    case SPS_TUNE_EXHAUSTIVE: s = run_exhaustive(pr, &best, res); break;
    default: return fail(SPS_ERR_INVALID_ARG, "unknown search algorithm");
  }
  if (s) return s;
  if (best.empty()) return fail(SPS_ERR_INVALID_ARG, "no evaluated configuration had a finite fitness");
  std::copy(best.begin(), best.end(), best_point);
  return SPS_OK;
}

sps_status space_problem(const sps_space* sp, Problem* pr) {
  if (!sp || sp->n_genes < 1 || !sp->n_values || !sp->kernel_of) return fail(SPS_ERR_INVALID_ARG, "bad space");
  pr->n_values.assign(sp->n_values, sp->n_values + sp->n_genes);
  for (int32_t g = 0; g < sp->n_genes; g++) {
    if (pr->n_values[g] < 1) return fail(SPS_ERR_INVALID_ARG, "every gene needs at least one value");
    if (g && sp->kernel_of[g] < sp->kernel_of[g - 1]) return fail(SPS_ERR_INVALID_ARG, "kernel_of must be non-decreasing");
    if (g == 0 || sp->kernel_of[g] != sp->kernel_of[g - 1]) pr->kernels.emplace_back();
    pr->kernels.back().push_back(g);
  }
  return SPS_OK;
}

// ------------------------------------------------------------------ plan space
// Gene value arrays (powers of two, Sec. 3.2) of each kernel kind.
const int32_t kU8Values[6][6] = {{1, 2, 4, 8}, {4, 8, 16, 32}, {1, 2, 4, 8, 16}, {1, 2, 4, 8, 16},
                                 {2, 4, 8, 16, 32, 64}, {0, 1, 2}};
const int32_t kU8Counts[6] = {4, 4, 5, 5, 6, 3};
const int32_t kStep2Values[5][6] = {{1, 2, 4, 8}, {4, 8, 16}, {1, 2, 4, 8, 16}, {1, 2, 4, 8, 16}, {1, 2, 4, 8, 16, 32}};
const int32_t kStep2Counts[5] = {4, 3, 5, 5, 6};
const int32_t kSnrValues[5] = {32, 64, 128, 256, 512};

struct PlanGene {
  int32_t kernel;            // 0 brute / step1, 1 step2 (subband), last: snr
  int32_t field;             // 0..5 dedispersion fields (5: presum), 6 snr threads
  std::vector<int32_t> values;
};

// The plan's genes.  The reduced space fixes all but six genes (subband mode:
// step one warps_dm and chunk; step two dms_per_thread, warps_dm and chunk;
// S/N threads) for 25 x 40 x 5 = 5000 points; in brute mode it keeps the
// brute kernel's first four genes (chunk 16) and the S/N threads.
std::vector<PlanGene> plan_genes(const sps_plan* p, int32_t which) {
  std::vector<PlanGene> out;
  auto u8 = [&](int32_t kernel, bool reduced_subband, bool reduced_brute) {
    for (int f = 0; f < 6; f++) {
      std::vector<int32_t> v(kU8Values[f], kU8Values[f] + kU8Counts[f]);
      if (reduced_subband) {
        const std::vector<std::vector<int32_t>> r = {{4}, {16}, {1, 2, 4, 8, 16}, {1}, {2, 4, 8, 16, 32}, {0}};
        v = r[f];
      } else if (reduced_brute) {
        const std::vector<std::vector<int32_t>> r = {{1, 2, 4, 8}, {4, 8, 16}, {1, 2, 4, 8, 16}, {1, 2}, {16}, {0, 1, 2}};
        v = r[f];
      }
      out.push_back({kernel, f, v});
    }
  };
  const bool red = which == SPS_SPACE_REDUCED;
  if (p->mode == SPS_MODE_BRUTE) {
    u8(0, false, red);
  } else {
    u8(0, red, false);
    for (int f = 0; f < 5; f++) {
      std::vector<int32_t> v(kStep2Values[f], kStep2Values[f] + kStep2Counts[f]);
      if (red) {
        const std::vector<std::vector<int32_t>> r = {{2, 4}, {8}, {1, 2, 4, 8, 16}, {1}, {1, 2, 4, 8}};
        v = r[f];
      }
      out.push_back({1, f, v});
    }
  }
  out.push_back({p->mode == SPS_MODE_BRUTE ? 1 : 2, 6, std::vector<int32_t>(kSnrValues, kSnrValues + 5)});
  return out;
}

sps_kernel_config point_config(const sps_plan* p, const std::vector<PlanGene>& genes, const int32_t* point) {
  sps_kernel_config c = p->cfg;
  for (size_t g = 0; g < genes.size(); g++) {
    const int32_t v = genes[g].values[point[g]];
    if (genes[g].field == 6) {
      c.snr.threads = v;
      continue;
    }
    sps_dedisp_config* k = p->mode == SPS_MODE_BRUTE ? &c.brute : (genes[g].kernel == 0 ? &c.step1 : &c.step2);
    int32_t* fields[6] = {&k->dms_per_thread, &k->samples_per_thread, &k->warps_dm, &k->warps_time, &k->chunk,
                          &k->presum};
    *fields[genes[g].field] = v;
  }
  return c;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" {

sps_status sps_optimize(const sps_space* space, const sps_search_desc* desc, sps_valid_fn valid,
                        sps_fitness_fn fitness, sps_trace_fn trace, void* user, int32_t* best_point,
                        sps_search_result* result) {
  clear_error();
  if (!fitness) return fail(SPS_ERR_INVALID_ARG, "null fitness callback");
  Problem pr;
  if (sps_status s = space_problem(space, &pr)) return s;
  pr.valid = [&](const Point& p) { return valid ? valid(p.data(), user) != 0 : true; };
  pr.fitness = [&](const Point& p) { return fitness(p.data(), user); };
  if (trace) pr.trace = [&](int64_t i, const Point& p, double f) { trace(i, p.data(), f, user); };
  return run_problem(pr, desc, best_point, result);
}

sps_status sps_tune_space(const sps_plan* p, int32_t which, int32_t max_genes, int32_t* n_genes,
                          int32_t* n_values, int32_t* kernel_of, int32_t* values) {
  clear_error();
  if (!p || !n_genes) return fail(SPS_ERR_INVALID_ARG, "null argument");
  const std::vector<PlanGene> genes = plan_genes(p, which);
  *n_genes = (int32_t)genes.size();
  if (!n_values) return SPS_OK;
  if (max_genes < (int32_t)genes.size()) return fail(SPS_ERR_INVALID_ARG, "max_genes too small");
  for (size_t g = 0; g < genes.size(); g++) {
    n_values[g] = (int32_t)genes[g].values.size();
    if (kernel_of) kernel_of[g] = genes[g].kernel;
    if (values)
      for (size_t v = 0; v < genes[g].values.size(); v++) values[g * SPS_TUNE_MAX_VALUES + v] = genes[g].values[v];
  }
  return SPS_OK;
}

sps_status sps_tune_config(const sps_plan* p, int32_t which, const int32_t* point, sps_kernel_config* out) {
  clear_error();
  if (!p || !point || !out) return fail(SPS_ERR_INVALID_ARG, "null argument");
  const std::vector<PlanGene> genes = plan_genes(p, which);
  for (size_t g = 0; g < genes.size(); g++)
    if (point[g] < 0 || point[g] >= (int32_t)genes[g].values.size())
      return fail(SPS_ERR_INVALID_ARG, "gene value index out of range");
  *out = point_config(p, genes, point);
  return check_config(p, *out, nullptr);
}

sps_status sps_tune(sps_plan* p, int32_t which, const sps_search_desc* desc, const uint8_t* x, int64_t x_pitch,
                    int32_t* D, void* workspace, size_t workspace_bytes, double* snr, int32_t* peak_t,
                    int32_t* peak_val, int32_t reps, double limit_ms, sps_trace_fn trace, void* user,
                    int32_t* best_point, sps_search_result* result, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_tune");
  if (!p || !desc || !best_point || !result) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (reps < 1) return fail(SPS_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  const std::vector<PlanGene> genes = plan_genes(p, which);
  const sps_kernel_config original = p->cfg;
  cudaEvent_t e0, e1;
  SPS_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SPS_ERR_CUDA, "cudaEventCreate");
  }
  sps_status hard = SPS_OK;  // an error that is not the configuration's fault stops the search
  std::string hard_msg;
  Problem pr;
  for (size_t g = 0; g < genes.size(); g++) {
    pr.n_values.push_back((int32_t)genes[g].values.size());
    if (g == 0 || genes[g].kernel != genes[g - 1].kernel) pr.kernels.emplace_back();
    pr.kernels.back().push_back((int32_t)g);
  }
  pr.valid = [&](const Point& pt) { return check_config(p, point_config(p, genes, pt.data()), nullptr) == SPS_OK; };
  // fitness: median over three trials of the mean time of `reps` back-to-back searches
  // A configuration the plan rejects, or whose workspace exceeds the one given,
  // scores +inf; a CUDA error stops the search.
  auto search_once = [&]() -> bool {
    const sps_status r = run_search(p, x, x_pitch, D, workspace, workspace_bytes, snr, peak_t, peak_val, nullptr, st);
    if (r == SPS_ERR_CUDA) {
      hard = r;
      hard_msg = sps_last_error();
    }
    return r == SPS_OK;
  };
  pr.fitness = [&](const Point& pt) -> double {
    if (hard) return kInf;
    if (apply_config(p, point_config(p, genes, pt.data())) != SPS_OK) return kInf;
    if (plan_workspace_bytes(p) > workspace_bytes) return kInf;
    if (!search_once()) return kInf;
    double trial[3];
    for (int t = 0; t < 3; t++) {
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps; r++)
        if (!search_once()) return kInf;
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        hard = SPS_ERR_CUDA;
        hard_msg = cudaGetErrorString(e);
        return kInf;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      trial[t] = (double)ms / reps;
    }
    std::sort(trial, trial + 3);
    return (limit_ms > 0.0 && trial[1] > limit_ms) ? kInf : trial[1];
  };
  if (trace) pr.trace = [&](int64_t i, const Point& pt, double f) { trace(i, pt.data(), f, user); };
  sps_status s = run_problem(pr, desc, best_point, result);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == SPS_OK && hard) s = fail(hard, "a launch failed during tuning: " + hard_msg);
  // leave the plan on the best configuration found (or where it was)
  if (s == SPS_OK && std::isfinite(result->best_fitness)) {
    s = apply_config(p, point_config(p, genes, best_point));
  } else {
    apply_config(p, original);
  }
  return s;
}

}  // extern "C"
