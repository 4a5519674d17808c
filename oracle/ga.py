"""Oracle of the auto-tuner: genetic algorithm, pure random search and exhaustive
search over a discrete parameter space -- TEST INFRASTRUCTURE ONLY.

Plain Python, written from the paper (Mikhailov & Sclocco, Sec. 3.1-3.2 and
Sec. 4) in its order and notation; the C++ tuner in the library shares no code
with it.  Both draw random numbers from the same counter-based generator,
SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), each implementing it from its
published definition, so that seeded runs can be compared draw for draw.

Readings of the paper taken here (the text does not fix them):
  * an individual is one value index per gene; genes are grouped by kernel;
  * initialisation draws every gene uniformly from its value array and redraws
    the whole individual until it satisfies the boundary conditions;
  * fitness is the measured pipeline time, lower is better; a failed or
    over-limit configuration gets +inf (the 3-minute penalty of Sec. 4);
  * tournament selection: a pool of N_pool = max(2, round(0.2 N_pop)) distinct
    individuals drawn by a partial Fisher-Yates shuffle; the fittest wins (ties:
    lower population index); repeated N_pop times;
  * pairing: the selected list is shuffled (Fisher-Yates) and taken in pairs;
    a pair of identical individuals swaps its second member with the first
    later individual that differs;
  * crossover per kernel with probability p_cross: uniform (each gene swapped
    when a draw exceeds 0.5, a swap that breaks a boundary condition undone) or
    one-point (a cut drawn in [0, n_k), the kernel's genes from the cut on
    swapped, undone if either offspring breaks a boundary condition);
  * mutation per kernel with probability p_mut: one gene of the kernel drawn
    uniformly gets a different value drawn uniformly; if that breaks a boundary
    condition the next values in cyclic order are tried, and the old value is
    kept if none is valid;
  * replacement: parents and offspring are ranked by (fitness, index) and the
    best N_pop/2 parents followed by the best N_pop/2 offspring form the next
    population; offspring left unevaluated because the budget ran out are not
    ranked, and further parents take their places;
  * renewal (Sec. 3.2 pairs individuals so that crossover yields new
    offspring; an offspring identical to an individual already evaluated is no
    new offspring either): after mutation, each offspring that repeats an
    evaluated individual or an earlier offspring of the same generation is
    mutated again -- a kernel drawn uniformly, then one of its genes, to a
    different valid value as in mutation -- up to `renew` times; renew = 0
    keeps every offspring as crossover and mutation left it;
  * the evaluation budget counts distinct evaluated individuals; repeats come
    from a cache; once the budget is spent further individuals score +inf;
  * pure random search draws valid individuals until the budget of distinct
    evaluations is spent; exhaustive search evaluates every valid point in
    lexicographic order (last gene fastest);
  * the end configurations of a run (Sec. 5, coefficient of variation): the
    GA's last population; for random search, which has no population, its last
    N_pop distinct evaluated individuals (the last "new random population").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    """Counter-based generator: output n = mix(seed + n * gamma), n = 1, 2, ..."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n): the top 53 bits as a fraction, times n."""
        return ((self.next_u64() >> 11) * n) >> 53

    def unit(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclass
class Space:
    n_values: list            # values per gene
    kernel_of: list           # kernel index per gene (non-decreasing)
    valid: object = None      # callable(point tuple) -> bool; None = all valid

    def __post_init__(self):
        # plain Python integers: the generator's arithmetic is exact big-integer math
        self.n_values = [int(v) for v in self.n_values]
        self.kernel_of = [int(k) for k in self.kernel_of]

    def kernels(self):
        out = {}
        for g, k in enumerate(self.kernel_of):
            out.setdefault(k, []).append(g)
        return [out[k] for k in sorted(out)]

    def is_valid(self, p) -> bool:
        return True if self.valid is None else bool(self.valid(tuple(p)))


@dataclass
class Result:
    best_point: tuple
    best_fitness: float
    evaluations: int
    generations: int
    trace: list = field(default_factory=list)       # (point, fitness) per distinct evaluation
    history: list = field(default_factory=list)     # (generation, evaluations, best fitness)
    final_population: list = field(default_factory=list)  # end configurations (Sec. 5)


class _Evaluator:
    def __init__(self, fitness, budget):
        self.fitness, self.budget = fitness, budget
        self.cache, self.trace = {}, []
        self.best_point, self.best = None, math.inf

    def __call__(self, p) -> float:
        p = tuple(p)
        if p in self.cache:
            return self.cache[p]
        if self.budget is not None and len(self.trace) >= self.budget:
            return math.inf
        f = float(self.fitness(p))
        self.cache[p] = f
        self.trace.append((p, f))
        if f < self.best:
            self.best, self.best_point = f, p
        return f

    @property
    def evaluations(self):
        return len(self.trace)


def random_valid_point(space: Space, rng: SplitMix64, max_tries: int = 1000):
    """Sec. 3.2: genes drawn uniformly from their value arrays, redrawn until valid."""
    for _ in range(max_tries):
        p = [rng.below(v) for v in space.n_values]
        if space.is_valid(p):
            return p
    raise RuntimeError("no valid individual found")


def tournament_pool_size(n_pop: int, pool_fraction: float) -> int:
    return min(n_pop, max(2, int(math.floor(pool_fraction * n_pop + 0.5))))


def _mutate_gene(space: Space, child, g, rng: SplitMix64):
    """One gene to a different value drawn uniformly; if that breaks a boundary
    condition the next values in cyclic order are tried, and the old value is
    kept if none is valid."""
    nv = space.n_values[g]
    if nv < 2:
        return
    old = child[g]
    v = rng.below(nv - 1)
    if v >= old:
        v += 1
    chosen = old
    for s in range(nv):
        cand = (v + s) % nv
        if cand == old:
            continue
        child[g] = cand
        if space.is_valid(child):
            chosen = cand
            break
    child[g] = chosen


def genetic(space: Space, fitness, n_pop=32, p_cross=0.8, p_mut=0.1, pool_fraction=0.2,
            crossover="uniform", max_evaluations=500, max_generations=1000, seed=1, renew=8) -> Result:
    """Sec. 3.2: initialise, evaluate, then select -> pair -> cross -> mutate ->
    (renew repeats) -> evaluate -> replace, until the evaluation budget or the
    generation limit."""
    if n_pop < 2 or n_pop % 2:
        raise ValueError("N_pop must be even and >= 2")
    rng = SplitMix64(seed)
    ev = _Evaluator(fitness, max_evaluations)
    kernels = space.kernels()
    n_pool = tournament_pool_size(n_pop, pool_fraction)

    population = [random_valid_point(space, rng) for _ in range(n_pop)]
    fit = [ev(p) for p in population]
    history = [(0, ev.evaluations, ev.best)]
    gen = 0
    while ev.evaluations < max_evaluations and gen < max_generations:
        gen += 1
        # selection: N_pop tournaments over pools of N_pool distinct individuals
        selected = []
        for _ in range(n_pop):
            idx = list(range(n_pop))
            for q in range(n_pool):
                r = q + rng.below(n_pop - q)
                idx[q], idx[r] = idx[r], idx[q]
            pool = idx[:n_pool]
            winner = min(pool, key=lambda j: (fit[j], j))
            selected.append(list(population[winner]))
        # pairing: shuffle, then avoid identical partners
        for q in range(n_pop - 1, 0, -1):
            r = rng.below(q + 1)
            selected[q], selected[r] = selected[r], selected[q]
        for q in range(0, n_pop, 2):
            if selected[q] == selected[q + 1]:
                for r in range(q + 2, n_pop):
                    if selected[r] != selected[q]:
                        selected[q + 1], selected[r] = selected[r], selected[q + 1]
                        break
        # crossover, per kernel, with probability p_cross
        offspring = [list(s) for s in selected]
        for q in range(0, n_pop, 2):
            a, b = offspring[q], offspring[q + 1]
            for genes in kernels:
                if rng.unit() < p_cross:
                    if crossover == "uniform":
                        for g in genes:
                            if rng.unit() > 0.5:
                                a[g], b[g] = b[g], a[g]
                                if not (space.is_valid(a) and space.is_valid(b)):
                                    a[g], b[g] = b[g], a[g]
                    else:
                        cut = rng.below(len(genes))
                        tail = genes[cut:]
                        for g in tail:
                            a[g], b[g] = b[g], a[g]
                        if not (space.is_valid(a) and space.is_valid(b)):
                            for g in tail:
                                a[g], b[g] = b[g], a[g]
        # mutation, per kernel, with probability p_mut
        for child in offspring:
            for genes in kernels:
                if rng.unit() < p_mut:
                    _mutate_gene(space, child, genes[rng.below(len(genes))], rng)
        # renewal: offspring that repeat an evaluated individual or an earlier
        # offspring of this generation mutate again, up to `renew` times each
        for j, child in enumerate(offspring):
            tries = 0
            while tries < renew and (tuple(child) in ev.cache or child in offspring[:j]):
                genes = kernels[rng.below(len(kernels))]
                _mutate_gene(space, child, genes[rng.below(len(genes))], rng)
                tries += 1
        off_fit = [ev(c) for c in offspring]
        # replacement: the fitter half of the parents and of the offspring; an
        # offspring left unevaluated because the budget ran out takes no place,
        # and the next-fittest parents fill the population instead
        evaluated = [j for j in range(n_pop) if tuple(offspring[j]) in ev.cache]
        off_rank = sorted(evaluated, key=lambda j: (off_fit[j], j))[: n_pop // 2]
        par_rank = sorted(range(n_pop), key=lambda j: (fit[j], j))[: n_pop - len(off_rank)]
        population = [population[j] for j in par_rank] + [offspring[j] for j in off_rank]
        fit = [fit[j] for j in par_rank] + [off_fit[j] for j in off_rank]
        history.append((gen, ev.evaluations, ev.best))
    return Result(ev.best_point, ev.best, ev.evaluations, gen, ev.trace, history,
                  [tuple(p) for p in population])


def random_search(space: Space, fitness, max_evaluations=500, seed=1, max_draws=None, n_pop=32) -> Result:
    """Sec. 4: new random individuals (no genetic operators) until the budget is spent."""
    rng = SplitMix64(seed)
    ev = _Evaluator(fitness, max_evaluations)
    draws = 0
    limit = max_draws if max_draws is not None else 100 * max_evaluations
    while ev.evaluations < max_evaluations and draws < limit:
        p = tuple(random_valid_point(space, rng))
        draws += 1
        if p in ev.cache:
            continue
        ev(p)
    return Result(ev.best_point, ev.best, ev.evaluations, 0, ev.trace, [(0, ev.evaluations, ev.best)],
                  [p for p, _ in ev.trace[-n_pop:]])


def coefficients_of_variation(end_configurations, values):
    """Sec. 5: for each gene, c_v = sigma / mu of the parameter's values over a
    run's end configurations (population standard deviation); None where the
    mean is zero (the paper leaves such a parameter out).  `values[g]` maps a
    gene's value index to the parameter value."""
    out = []
    for g in range(len(values)):
        v = [values[g][p[g]] for p in end_configurations]
        mu = sum(v) / len(v)
        if mu == 0:
            out.append(None)
            continue
        var = sum((a - mu) ** 2 for a in v) / len(v)
        out.append(math.sqrt(var) / mu)
    return out


def exhaustive(space: Space, fitness) -> Result:
    """Every valid point, lexicographic order (last gene fastest)."""
    ev = _Evaluator(fitness, None)
    p = [0] * len(space.n_values)
    while True:
        if space.is_valid(p):
            ev(p)
        g = len(p) - 1
        while g >= 0:
            p[g] += 1
            if p[g] < space.n_values[g]:
                break
            p[g] = 0
            g -= 1
        if g < 0:
            break
    return Result(ev.best_point, ev.best, ev.evaluations, 0, ev.trace, [(0, ev.evaluations, ev.best)])
