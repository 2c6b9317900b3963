// Host side of the amplitude engine: random grid circuits, the complex
// graphical model (paper Sec. III), elimination orders, slicing and the step
// list of bucket elimination (Sec. IV, App. A), and the device layout the
// kernels in exec.cu consume.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <cstddef>
#include <numeric>

#include "host.h"

namespace qgm {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

// ---------------------------------------------------------------- circuit
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): golden-ratio increment and
// two xor-shift-multiply rounds.
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// The 8 CZ layers [HZ0, HZ2, VT0, VT2, HZ1, HZ3, VT1, VT3]: HZ_o pairs
// (r,c)-(r,c+1) when c = o + 2(r mod 2) (mod 4); VT_o pairs (r,c)-(r+1,c)
// when r = o + 2(c mod 2) (mod 4).
static std::vector<std::vector<std::pair<int, int>>> cz_patterns(int rows, int cols) {
  auto hz = [&](int o) {
    std::vector<std::pair<int, int>> v;
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c + 1 < cols; ++c)
        if (c % 4 == (o + 2 * (r % 2)) % 4) v.push_back({r * cols + c, r * cols + c + 1});
    return v;
  };
  auto vt = [&](int o) {
    std::vector<std::pair<int, int>> v;
    for (int r = 0; r + 1 < rows; ++r)
      for (int c = 0; c < cols; ++c)
        if (r % 4 == (o + 2 * (c % 2)) % 4) v.push_back({r * cols + c, (r + 1) * cols + c});
    return v;
  };
  return {hz(0), hz(2), vt(0), vt(2), hz(1), hz(3), vt(1), vt(3)};
}

static Circuit grid_circuit(int rows, int cols, int depth, uint64_t seed, int param) {
  Circuit c;
  c.n = rows * cols;
  c.rows = rows;
  c.cols = cols;
  c.depth = depth;
  c.seed = seed;
  c.param = param;
  const int n = c.n;
  auto pats = cz_patterns(rows, cols);
  SplitMix64 rng(seed);
  for (int q = 0; q < n; ++q) c.gates.push_back({QGM_GATE_H, 0, q, -1, 0.0, 0.0});
  std::vector<char> prev(n, 0), had_t(n, 0);
  for (int t = 1; t < depth; ++t) {
    std::vector<char> in_cz(n, 0);
    for (auto &pr : pats[(t - 1) % 8]) {
      c.gates.push_back({QGM_GATE_CZ, t, pr.first, pr.second, 0.0, 0.0});
      in_cz[pr.first] = in_cz[pr.second] = 1;
    }
    for (int q = 0; q < n; ++q) {
      if (!(prev[q] && !in_cz[q])) continue;
      if (!had_t[q]) {
        had_t[q] = 1;
        c.gates.push_back({QGM_GATE_T, t, q, -1, 0.0, 0.0});
      } else if (param) {
        double th = M_PI * rng.uniform();
        double ph = 2.0 * M_PI * rng.uniform();
        c.param_gates.push_back((int)c.gates.size());
        c.gates.push_back({QGM_GATE_RXY, t, q, -1, th, ph});
      } else {
        uint64_t r = rng.next();
        c.gates.push_back({(r >> 63) == 0 ? QGM_GATE_X12 : QGM_GATE_Y12, t, q, -1, 0.0, 0.0});
      }
    }
    prev = in_cz;
  }
  return c;
}

// ------------------------------------------------------------------ model
// psi_U(b', b) = <b'|U|b>; the non-diagonal fixed gates are stored with the
// common 2^{-1/2} pulled out (entries in {+-1, +-i}), tracked by half_pow.
static void gate_table(const qgm_gate &g, cd t[4], int *half_pow) {
  const cd I(0.0, 1.0);
  *half_pow = 0;
  switch (g.kind) {
    case QGM_GATE_H: t[0] = 1; t[1] = 1; t[2] = 1; t[3] = -1; *half_pow = 1; break;
    case QGM_GATE_X12: t[0] = 1; t[1] = -I; t[2] = -I; t[3] = 1; *half_pow = 1; break;
    case QGM_GATE_Y12: t[0] = 1; t[1] = -1; t[2] = 1; t[3] = 1; *half_pow = 1; break;
    case QGM_GATE_RXY: {
      double c = std::cos(g.theta / 2), s = std::sin(g.theta / 2);
      t[0] = c;
      t[1] = -I * std::exp(-I * g.phi) * s;
      t[2] = -I * std::exp(I * g.phi) * s;
      t[3] = c;
      break;
    }
    case QGM_GATE_T: t[0] = 1; t[1] = std::exp(I * (M_PI / 4)); break;
    case QGM_GATE_CZ: t[0] = 1; t[1] = 1; t[2] = 1; t[3] = -1; break;
  }
}

static int build_model(const Circuit &c, Model &m) {
  m = Model();
  m.n = c.n;
  m.rows = c.rows;
  m.cols = c.cols;
  m.gates = c.gates;
  std::vector<int> cur(c.n);
  for (int q = 0; q < c.n; ++q) {
    cur[q] = q;
    m.var_qubit.push_back(q);
    m.var_k.push_back(0);
    m.inputs.push_back(q);
  }
  int nv = c.n;
  for (size_t gi = 0; gi < c.gates.size(); ++gi) {
    const qgm_gate &g = c.gates[gi];
    MFactor f;
    f.gate = (int)gi;
    gate_table(g, f.t, &f.half_pow);
    if (g.kind == QGM_GATE_CZ) {
      f.nv = 2;
      f.v[0] = cur[g.q0];
      f.v[1] = cur[g.q1];
    } else if (g.kind == QGM_GATE_T) {
      f.nv = 1;
      f.v[0] = cur[g.q0];
    } else {
      int v = nv++;
      m.var_qubit.push_back(g.q0);
      m.var_k.push_back(m.var_k[cur[g.q0]] + 1);
      f.nv = 2;
      f.v[0] = v;  // b' (after the gate)
      f.v[1] = cur[g.q0];
      cur[g.q0] = v;
      m.L++;
      if (g.kind == QGM_GATE_RXY) m.param_factor.push_back((int)m.factors.size());
    }
    m.factors.push_back(f);
  }
  m.n_vars = nv;
  m.outputs = cur;
  return QGM_OK;
}

// ------------------------------------------------------------------- plan
static std::vector<int> qubit_rank(int rows, int cols, bool transpose) {
  bool colmajor = rows < cols;
  if (transpose) colmajor = !colmajor;
  std::vector<int> rank(rows * cols);
  for (int q = 0; q < rows * cols; ++q) {
    int r = q / cols, c = q % cols;
    rank[q] = colmajor ? c * rows + r : q;
  }
  return rank;
}

// Table of a factor re-laid out over `scope` (C-order), given its current
// scope and table.  `scope` must contain every variable of `from`.
static std::vector<cd> expand_table(const std::vector<int> &from_scope, const std::vector<cd> &from,
                                    const std::vector<int> &scope) {
  const int r = (int)scope.size();
  std::vector<int> where(from_scope.size());
  for (size_t a = 0; a < from_scope.size(); ++a)
    where[a] = (int)(std::find(scope.begin(), scope.end(), from_scope[a]) - scope.begin());
  std::vector<cd> out((size_t)1 << r);
  const int fr = (int)from_scope.size();
  for (size_t i = 0; i < out.size(); ++i) {
    size_t fi = 0;
    for (int a = 0; a < fr; ++a) fi |= ((i >> (r - 1 - where[a])) & 1) << (fr - 1 - a);
    out[i] = from[fi];
  }
  return out;
}

// Fix the input variables to 0, then merge factors with equal scopes and
// absorb factors whose scope is a subset of another's (the product is the
// same function; fewer, larger tables).
static void reduce_factors(const Model &m, std::vector<LeafFactor> &leaves, cd &constant,
                           int &half_pow_total) {
  std::vector<char> is_in(m.n_vars, 0);
  for (int v : m.inputs) is_in[v] = 1;
  leaves.clear();
  constant = 1.0;
  half_pow_total = 0;
  std::map<std::vector<int>, int> by_scope;
  for (size_t fi = 0; fi < m.factors.size(); ++fi) {
    const MFactor &f = m.factors[fi];
    half_pow_total += f.half_pow;
    std::vector<int> sc;
    std::vector<cd> tab;
    // substitute inputs = 0
    std::vector<int> keep;
    for (int a = 0; a < f.nv; ++a)
      if (!is_in[f.v[a]]) keep.push_back(a);
    for (int a : keep) sc.push_back(f.v[a]);
    tab.assign((size_t)1 << keep.size(), 0.0);
    for (size_t i = 0; i < tab.size(); ++i) {
      int full = 0;
      for (size_t b = 0; b < keep.size(); ++b)
        if ((i >> (keep.size() - 1 - b)) & 1) full |= 1 << (f.nv - 1 - keep[b]);
      tab[i] = f.t[full];
    }
    if (sc.empty()) {
      constant *= tab[0];
      continue;
    }
    // canonical: scope sorted by var id (merging two equal vars is impossible
    // here: a two-variable factor always has two distinct variables)
    std::vector<int> sorted = sc;
    std::sort(sorted.begin(), sorted.end());
    std::vector<cd> st = expand_table(sc, tab, sorted);
    auto it = by_scope.find(sorted);
    if (it != by_scope.end()) {
      LeafFactor &L = leaves[it->second];
      for (size_t i = 0; i < st.size(); ++i) L.table[i] *= st[i];
      L.members.push_back((int)fi);
    } else {
      by_scope[sorted] = (int)leaves.size();
      LeafFactor L;
      L.scope = sorted;
      L.table = st;
      L.members.push_back((int)fi);
      leaves.push_back(L);
    }
  }
  // absorb proper subsets into the first superset
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t a = 0; a < leaves.size() && !changed; ++a) {
      for (size_t b = 0; b < leaves.size(); ++b) {
        if (a == b || leaves[a].scope.size() >= leaves[b].scope.size()) continue;
        if (!std::includes(leaves[b].scope.begin(), leaves[b].scope.end(), leaves[a].scope.begin(),
                           leaves[a].scope.end()))
          continue;
        std::vector<cd> ex = expand_table(leaves[a].scope, leaves[a].table, leaves[b].scope);
        for (size_t i = 0; i < ex.size(); ++i) leaves[b].table[i] *= ex[i];
        leaves[b].members.insert(leaves[b].members.end(), leaves[a].members.begin(),
                                 leaves[a].members.end());
        leaves.erase(leaves.begin() + a);
        changed = true;
        break;
      }
    }
  }
}

struct Graph {
  int nv;
  int words;
  std::vector<uint64_t> bits;  // adjacency bitsets
  std::vector<char> alive;
  explicit Graph(int n) : nv(n), words((n + 63) / 64), bits((size_t)n * ((n + 63) / 64), 0), alive(n, 0) {}
  uint64_t *row(int v) { return &bits[(size_t)v * words]; }
  bool has(int a, int b) { return (row(a)[b >> 6] >> (b & 63)) & 1; }
  void add(int a, int b) {
    row(a)[b >> 6] |= 1ULL << (b & 63);
    row(b)[a >> 6] |= 1ULL << (a & 63);
  }
  int degree(int v) {
    int d = 0;
    uint64_t *r = row(v);
    for (int w = 0; w < words; ++w) d += __builtin_popcountll(r[w]);
    return d;
  }
  std::vector<int> nbrs(int v) {
    std::vector<int> out;
    uint64_t *r = row(v);
    for (int w = 0; w < words; ++w) {
      uint64_t x = r[w];
      while (x) {
        int b = __builtin_ctzll(x);
        out.push_back(w * 64 + b);
        x &= x - 1;
      }
    }
    return out;
  }
  // eliminate v: neighbours become a clique; returns the clique size (v + nbrs)
  int eliminate(int v) {
    std::vector<int> nb = nbrs(v);
    for (size_t i = 0; i < nb.size(); ++i)
      for (size_t j = i + 1; j < nb.size(); ++j) add(nb[i], nb[j]);
    for (int a : nb) row(a)[v >> 6] &= ~(1ULL << (v & 63));
    std::fill(row(v), row(v) + words, 0);
    alive[v] = 0;
    return 1 + (int)nb.size();
  }
  int fill(int v) {
    std::vector<int> nb = nbrs(v);
    int f = 0;
    for (size_t i = 0; i < nb.size(); ++i)
      for (size_t j = i + 1; j < nb.size(); ++j)
        if (!has(nb[i], nb[j])) ++f;
    return f;
  }
};

// Interaction graph (Sec. III.B) on the variables in `in_graph`.
static Graph make_graph(const qgm_plan *p, const std::vector<char> &in_graph) {
  Graph g(p->model.n_vars);
  for (int v = 0; v < p->model.n_vars; ++v) g.alive[v] = in_graph[v];
  for (const LeafFactor &L : p->leaves)
    for (size_t a = 0; a < L.scope.size(); ++a)
      for (size_t b = a + 1; b < L.scope.size(); ++b)
        if (in_graph[L.scope[a]] && in_graph[L.scope[b]]) g.add(L.scope[a], L.scope[b]);
  return g;
}

// Min-fill: repeatedly eliminate the vertex adding the fewest fill edges;
// ties by fewest neighbours, then smallest id.  Vertices in `keep` stay.
static std::vector<int> order_minfill(Graph g, const std::vector<char> &keep) {
  std::vector<int> order;
  std::vector<int> fillc(g.nv, -1);
  std::vector<char> dirty(g.nv, 1);
  while (true) {
    int best = -1, bf = 0, bd = 0;
    for (int v = 0; v < g.nv; ++v) {
      if (!g.alive[v] || keep[v]) continue;
      if (dirty[v]) {
        fillc[v] = g.fill(v);
        dirty[v] = 0;
      }
      int f = fillc[v], d = g.degree(v);
      if (best < 0 || f < bf || (f == bf && d < bd)) {
        best = v;
        bf = f;
        bd = d;
      }
    }
    if (best < 0) break;
    // fill counts change for vertices within distance 2 of `best`
    std::vector<int> nb = g.nbrs(best);
    for (int a : nb) {
      dirty[a] = 1;
      for (int b : g.nbrs(a)) dirty[b] = 1;
    }
    g.eliminate(best);
    for (int a : nb)
      for (int b : g.nbrs(a)) dirty[b] = 1;
    order.push_back(best);
  }
  return order;
}

static std::vector<int> order_vertical(const qgm_plan *p, const std::vector<char> &elim, bool transpose) {
  const Model &m = p->model;
  int rows = m.rows ? m.rows : 1, cols = m.rows ? m.cols : m.n;
  std::vector<int> rank = qubit_rank(rows, cols, transpose);
  std::vector<int> vs;
  for (int v = 0; v < m.n_vars; ++v)
    if (elim[v]) vs.push_back(v);
  std::sort(vs.begin(), vs.end(), [&](int a, int b) {
    int ra = rank[m.var_qubit[a]], rb = rank[m.var_qubit[b]];
    if (ra != rb) return ra < rb;
    if (m.var_k[a] != m.var_k[b]) return m.var_k[a] < m.var_k[b];
    return a < b;
  });
  return vs;
}

// ---------------------------------------------------------- arena allocator
struct Arena {
  std::map<int64_t, int64_t> free_;  // off -> size
  int64_t top = 0, peak = 0;
  int64_t al = 256;
  int64_t align(int64_t x) const { return (x + al - 1) & ~(al - 1); }
  int64_t alloc(int64_t bytes) {
    bytes = align(std::max<int64_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        int64_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        return off;
      }
    }
    int64_t off = top;
    top += bytes;
    peak = std::max(peak, top);
    return off;
  }
  void release(int64_t off, int64_t bytes) {
    bytes = align(std::max<int64_t>(bytes, 1));
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == top) {
      top = it->first;
      free_.erase(it);
    }
  }
};

// Symbolic bucket elimination (App. A) for `order` with `slice` variables
// removed: the step list, its algorithmic bytes/flops and the arena peak.
static SimResult simulate(const qgm_plan *p, const std::vector<int> &order_in,
                          const std::vector<char> &sliced, int max_fuse, bool want_steps) {
  const Model &m = p->model;
  SimResult R;
  std::vector<int> order;
  for (int v : order_in)
    if (!sliced[v]) order.push_back(v);
  const int ne = (int)order.size();
  std::vector<int> pos(m.n_vars, -1);
  for (int i = 0; i < ne; ++i) pos[order[i]] = i;
  // open variables after the eliminated ones, qubit n-1 first, so that the
  // final tensor's index has qubit j at bit j
  for (size_t i = 0; i < p->open_vars.size(); ++i) pos[p->open_vars[i]] = ne + (int)i;
  const int64_t Bp = p->Bp;

  auto entries = [&](const SymTensor &t) {
    return ((int64_t)1 << t.vars.size()) * (t.batched ? Bp : 1);
  };
  std::vector<SymTensor> &T = R.tensors;
  std::vector<std::vector<int>> bucket(ne);
  std::vector<int> live(m.n_vars, 0);
  std::vector<int> finals;
  Arena arena;

  auto place = [&](int id) {
    const SymTensor &t = T[id];
    if (t.vars.empty() || pos[t.vars[0]] >= ne)
      finals.push_back(id);
    else
      bucket[pos[t.vars[0]]].push_back(id);
    for (int v : t.vars) live[v]++;
  };
  for (size_t li = 0; li < p->leaves.size(); ++li) {
    const LeafFactor &L = p->leaves[li];
    SymTensor t;
    t.leaf = (int)li;
    for (int v : L.scope) {
      int role = p->var_role[v];
      if (role == 2) t.batched = true;
      if (pos[v] >= 0) t.vars.push_back(v);
    }
    std::sort(t.vars.begin(), t.vars.end(), [&](int a, int b) { return pos[a] < pos[b]; });
    t.entries = entries(t);
    T.push_back(t);
    place((int)T.size() - 1);
  }
  const bool trees = p->trees_ok;
  const bool nest = p->nest_ok;
  int n_meta = 0;
  auto by_pos = [&](int a, int b) { return pos[a] < pos[b]; };
  // One step: out = sum over `summed` of the product of the inputs.  The
  // step's union lists the summed variables first, then the kept ones, each
  // in elimination order; the output keeps the kept ones in that order.
  auto emit = [&](std::vector<int> inputs, std::vector<int> summed, bool gemm = false, int k_inner = 0,
                  std::vector<char> inner = {}) -> int {
    std::vector<int> all;
    bool batched = false;
    for (int id : inputs) {
      for (int v : T[id].vars) all.push_back(v);
      batched |= T[id].batched;
    }
    std::sort(all.begin(), all.end(), by_pos);
    all.erase(std::unique(all.begin(), all.end()), all.end());
    // summed variables in elimination order; a nested step keeps its inner
    // ones (the last k_inner) after the outer ones
    std::sort(summed.begin(), summed.end() - k_inner, by_pos);
    std::sort(summed.end() - k_inner, summed.end(), by_pos);
    std::vector<int> uni = summed;
    for (int v : all)
      if (std::find(summed.begin(), summed.end(), v) == summed.end()) uni.push_back(v);
    const int k = (int)summed.size();
    SymTensor out;
    out.vars.assign(uni.begin() + k, uni.end());
    out.batched = batched;
    out.entries = entries(out);
    out.meta = n_meta++;
    out.off = arena.alloc(out.entries * 8);
    StepRec s;
    s.inputs = inputs;
    s.uni = uni;
    s.k = k;
    s.batched = batched;
    double rb = 0;
    for (int id : inputs) {
      rb += (double)T[id].entries * 8;
      for (int v : T[id].vars) live[v]--;
      if (T[id].leaf < 0) arena.release(T[id].off, T[id].entries * 8);
    }
    s.bytes = rb + (double)out.entries * 8;
    s.flops = (double)out.entries * (double)(1LL << k) * (6.0 * (inputs.size() - 1) + 2.0);
    R.bytes += s.bytes;
    R.flops += s.flops;
    R.max_step_bytes = std::max(R.max_step_bytes, s.bytes);
    R.max_entries = std::max(R.max_entries, out.entries);
    T.push_back(out);
    int oid = (int)T.size() - 1;
    s.out = oid;
    s.gemm = gemm;
    s.k_inner = k_inner;
    s.inner = inner;
    if (!want_steps) {
      s.inputs.clear();
      s.uni.clear();
      s.inner.clear();
    }
    R.steps.push_back(s);
    return oid;
  };
  // an intermediate consumed inside the same bucket holds its variables live
  auto hold = [&](int id) {
    for (int v : T[id].vars) live[v]++;
    return id;
  };
  // more than MAXIN inputs: multiply the smallest ones together first
  auto shrink = [&](std::vector<int> &inputs) {
    while ((int)inputs.size() > MAXIN) {
      std::stable_sort(inputs.begin(), inputs.end(),
                       [&](int a, int b) { return T[a].entries < T[b].entries; });
      std::vector<int> two = {inputs[0], inputs[1]};
      inputs.erase(inputs.begin(), inputs.begin() + 2);
      inputs.push_back(hold(emit(two, {})));
    }
  };
  auto holds = [&](int id, int v) {
    return std::find(T[id].vars.begin(), T[id].vars.end(), v) != T[id].vars.end();
  };
  // One contraction (a bucket, or a node of a bucket's contraction tree).
  // GEMM-shaped: the two largest inputs hold every summed variable and every
  // other input fits inside one of them (it is multiplied into that operand
  // first, a product step with nothing summed).
  auto contract = [&](std::vector<int> inputs, const std::vector<int> &summed) -> int {
    shrink(inputs);
    const int k = (int)summed.size();
    if (p->gemm_ok && k >= (p->gemm_tc ? 2 : 4) && inputs.size() >= 2) {
      std::vector<int> by = inputs;
      std::stable_sort(by.begin(), by.end(), [&](int a, int b) { return T[a].vars.size() > T[b].vars.size(); });
      const int A = by[0], Bt = by[1];
      bool ok = T[A].vars.size() >= 10 && T[Bt].vars.size() >= 10;
      for (int v : summed) ok = ok && holds(A, v) && holds(Bt, v);
      std::vector<int> toA = {A}, toB = {Bt};
      for (size_t q = 2; q < by.size() && ok; ++q) {
        bool inA = true, inB = true;
        for (int v : T[by[q]].vars) {
          inA = inA && holds(A, v);
          inB = inB && holds(Bt, v);
        }
        if (T[by[q]].vars.size() > 8 || (!inA && !inB)) ok = false;
        else if (inB && (!inA || T[Bt].entries < T[A].entries)) toB.push_back(by[q]);
        else toA.push_back(by[q]);
      }
      int nm = 0, nn = 0, ns = 0;
      std::vector<int> kept;
      for (int id : inputs)
        for (int v : T[id].vars)
          if (std::find(summed.begin(), summed.end(), v) == summed.end() &&
              std::find(kept.begin(), kept.end(), v) == kept.end())
            kept.push_back(v);
      for (int v : kept) {
        if (!ok) break;
        const bool ha = holds(A, v), hb = holds(Bt, v);
        if (!ha && !hb) ok = false;
        nm += ha && !hb;
        nn += hb && !ha;
        ns += ha && hb;
      }
      // the shared kept variables index independent products (a grid
      // dimension of the launch): at most 15 of them
      if (ns > 15) ok = false;
      // FP32-core kernel: tiles of 64 x 64 or, with a wide batch (many GEMMs
      // per launch), 64 x 32 outputs, the operand with six or more private
      // kept variables first, 16 summed entries per chunk
      const int min_side = Bp >= 64 ? 5 : 6;
      const bool fp32_ok = k >= 4 && std::max(nm, nn) >= 6 && std::min(nm, nn) >= min_side;
      // tensor cores: whenever the step's tensor-core form exists (fewer than
      // 16 summed entries are padded with zeros to one chunk, worth it only
      // for large outputs)
      bool tc_ok = false;
      if (ok && p->gemm_tc && !fp32_ok) {
        GemmDesc tg{};
        tg.nm = nm;
        tg.nn = nn;
        tg.nk = k;
        tg.ns = ns;
        for (int id : toA) tg.a_bat |= T[id].batched ? 1 : 0;
        for (int id : toB) tg.b_bat |= T[id].batched ? 1 : 0;
        tg.o_bat = tg.a_bat | tg.b_bat;
        const double out_entries = std::ldexp(tg.o_bat ? (double)Bp : 1.0, nm + nn + ns);
        tc_ok = tc_config(tg, (int)Bp, 4).ok && (k >= 4 || out_entries >= 1048576.0);
      }
      if (ok && (fp32_ok || tc_ok) && nm < GMAXB && nn < GMAXB) {
        auto premul = [&](std::vector<int> &grp) { return grp.size() == 1 ? grp[0] : hold(emit(grp, {})); };
        const int a2 = premul(toA), b2 = premul(toB);
        const bool a_first = fp32_ok ? nm >= 6 : nm >= nn;
        return a_first ? emit({a2, b2}, summed, true) : emit({b2, a2}, summed, true);
      }
    }
    if (nest && inputs.size() >= 3 && k >= 2) {
      // Nested product-sum: split the inputs into an inner group G2 and an
      // outer group G1 so that the summed variables held by G2 only (K2) are
      // summed in an inner loop: sum_K1 prod(G1) * sum_K2 prod(G2).  Inputs
      // inside the largest member of their group are multiplied into it
      // first.  Cost per output entry, in complex products:
      // 2^|K1| (2^|K2| m2 + m1) against 2^|K| m for the flat product-sum.
      const int n = (int)inputs.size();
      int64_t out_vars = 0;
      std::vector<int> allv;
      for (int id : inputs)
        for (int v : T[id].vars)
          if (std::find(allv.begin(), allv.end(), v) == allv.end()) allv.push_back(v);
      out_vars = (int64_t)allv.size() - k;
      bool bat = false;
      for (int id : inputs) bat |= T[id].batched;
      const double bf = bat ? (double)Bp : 1.0;
      auto group_plan = [&](const std::vector<int> &grp, std::vector<std::vector<int>> &parts) {
        // members inside the group's largest member are multiplied into it
        parts.clear();
        if (grp.empty()) return 0.0;
        int big = grp[0];
        for (int id : grp)
          if (T[id].vars.size() > T[big].vars.size()) big = id;
        std::vector<int> into = {big};
        for (int id : grp) {
          if (id == big) continue;
          bool inside = true;
          for (int v : T[id].vars) inside = inside && holds(big, v);
          if (inside) into.push_back(id);
          else parts.push_back({id});
        }
        parts.insert(parts.begin(), into);
        return into.size() > 1 ? std::ldexp(bf, (int)T[big].vars.size()) * (double)into.size() : 0.0;
      };
      const double flat = std::ldexp(bf, (int)(out_vars + k)) * n;
      double best = 0.7 * flat;
      int best_mask = 0;
      for (int mask = 1; mask < (1 << n) - 1; ++mask) {
        std::vector<int> g1, g2;
        for (int i = 0; i < n; ++i) ((mask >> i) & 1 ? g2 : g1).push_back(inputs[i]);
        int k2 = 0;
        for (int v : summed) {
          bool in1 = false, in2 = false;
          for (int id : g1) in1 = in1 || holds(id, v);
          for (int id : g2) in2 = in2 || holds(id, v);
          k2 += in2 && !in1;
        }
        if (k2 == 0 || k2 == k) continue;
        std::vector<std::vector<int>> p1, p2;
        const double pre = group_plan(g1, p1) + group_plan(g2, p2);
        const double cost =
            std::ldexp(bf, (int)(out_vars + k - k2)) * ((double)((int64_t)1 << k2) * (double)p2.size() + (double)p1.size()) +
            pre;
        if (cost < best && flat - cost >= std::ldexp(bf, 12)) {
          best = cost;
          best_mask = mask;
        }
      }
      if (best_mask) {
        std::vector<int> g1, g2;
        for (int i = 0; i < n; ++i) ((best_mask >> i) & 1 ? g2 : g1).push_back(inputs[i]);
        std::vector<int> k1v, k2v;
        for (int v : summed) {
          bool in1 = false;
          for (int id : g1) in1 = in1 || holds(id, v);
          (in1 ? k1v : k2v).push_back(v);
        }
        std::vector<std::vector<int>> p1, p2;
        group_plan(g1, p1);
        group_plan(g2, p2);
        std::vector<int> ins;
        std::vector<char> inner;
        for (int side = 0; side < 2; ++side)
          for (auto &part : side ? p2 : p1) {
            ins.push_back(part.size() == 1 ? part[0] : hold(emit(part, {})));
            inner.push_back((char)side);
          }
        std::vector<int> sm = k1v;
        sm.insert(sm.end(), k2v.begin(), k2v.end());
        return emit(ins, sm, false, (int)k2v.size(), inner);
      }
    }
    return emit(inputs, summed);
  };
  // Contraction tree of a bucket with three or more inputs (App. A sums the
  // bucket's product in one go; multiplying pairs first and summing each
  // variable as soon as no other factor holds it gives the same sum with
  // fewer products).  Dynamic programming over subsets of the inputs for the
  // cheapest binary tree (cost of a node: entries of its union plus entries
  // written; intermediates at most one variable wider than the widest input
  // or the output), then children whose union lies inside the parent's are
  // merged back into it when that is cheaper.  Used when it beats the single
  // product-sum by a clear margin.
  auto contract_tree = [&](std::vector<int> inputs, const std::vector<int> &uni, int k) -> int {
    const int n = (int)inputs.size(), U = (int)uni.size();
    std::vector<int> summed(uni.begin(), uni.begin() + k);
    if (!trees || n < 3 || n > MAXIN || U > 62) return contract(inputs, summed);
    std::vector<uint64_t> vm(n);
    int widest = 0;
    for (int i = 0; i < n; ++i) {
      for (int v : T[inputs[i]].vars) vm[i] |= 1ull << (std::find(uni.begin(), uni.end(), v) - uni.begin());
      widest = std::max(widest, (int)T[inputs[i]].vars.size());
    }
    const uint64_t smask = (k >= 64) ? ~0ull : ((1ull << k) - 1);
    const int full = (1 << n) - 1;
    std::vector<uint64_t> all(full + 1, 0), res(full + 1, 0);
    std::vector<char> bat(full + 1, 0);
    for (int t = 1; t <= full; ++t) {
      const int i = __builtin_ctz(t);
      all[t] = all[t & (t - 1)] | vm[i];
      bat[t] = bat[t & (t - 1)] | (T[inputs[i]].batched ? 1 : 0);
    }
    for (int t = 1; t <= full; ++t) res[t] = all[t] & ~(smask & ~all[full ^ t]);
    // variables of a child as its parent sees them: a node's result, but an
    // input itself (nothing is summed inside a single input)
    std::vector<uint64_t> cv(full + 1, 0);
    for (int t = 1; t <= full; ++t) cv[t] = (t & (t - 1)) ? res[t] : all[t];
    const int limit = std::max(widest, __builtin_popcountll(res[full])) + 1;
    auto ent = [&](uint64_t mask, bool b) { return std::ldexp(b ? (double)Bp : 1.0, __builtin_popcountll(mask)); };
    const double step_over = 256.0;
    std::vector<double> best(full + 1, 0.0);
    std::vector<int> split_of(full + 1, 0);
    for (int t = 1; t <= full; ++t) {
      if (!(t & (t - 1))) continue;
      best[t] = 1e300;
      if (t != full && __builtin_popcountll(res[t]) > limit) continue;
      const int low = t & -t, rest = t ^ low;
      // t1 = low + any proper subset of the rest (t2 non-empty)
      for (int sub = (rest - 1) & rest;; sub = (sub - 1) & rest) {
        const int t1 = low | sub, t2 = t ^ t1;
        if (best[t1] < 1e299 && best[t2] < 1e299) {
          const double c = best[t1] + best[t2] + ent(cv[t1] | cv[t2], bat[t]) + ent(res[t], bat[t]) + step_over;
          if (c < best[t]) {
            best[t] = c;
            split_of[t] = t1;
          }
        }
        if (sub == 0) break;
      }
    }
    const double fused = (n - 1) * ent(all[full], bat[full]) + ent(res[full], bat[full]) + step_over;
    // only where it saves a clear share and a sizeable amount of work: small
    // buckets stay one step (each extra step has a fixed cost)
    if (!(best[full] < 0.8 * fused) || fused - best[full] < ent(0xfffull, bat[full]))
      return contract(inputs, summed);
    // emit the tree: a leaf is an input, a node a subset of the inputs; a
    // child is merged into its parent when the parent's union covers it and
    // that is cheaper
    std::function<int(int)> run = [&](int t) -> int {
      if (!(t & (t - 1))) return inputs[__builtin_ctz(t)];
      // flatten children whose contraction is better done inside this node
      std::vector<int> kids = {split_of[t], t ^ split_of[t]};
      const uint64_t u = cv[split_of[t]] | cv[t ^ split_of[t]];
      bool changed = true;
      while (changed) {
        changed = false;
        for (size_t q = 0; q < kids.size(); ++q) {
          const int c = kids[q];
          if (!(c & (c - 1))) continue;
          const uint64_t uc = cv[split_of[c]] | cv[c ^ split_of[c]];
          if (uc & ~u) continue;
          const double sep = ent(uc, bat[c]) + ent(res[c], bat[c]) + step_over;
          if (ent(u, bat[t]) <= sep) {
            kids[q] = split_of[c];
            kids.push_back(c ^ split_of[c]);
            changed = true;
            break;
          }
        }
      }
      std::vector<int> ins;
      for (int c : kids) {
        const int id = run(c);
        ins.push_back((c & (c - 1)) ? hold(id) : id);
      }
      std::vector<int> sm;
      uint64_t gone = 0;
      for (int c : kids) gone |= cv[c];
      gone &= ~res[t];
      for (int b = 0; b < U; ++b)
        if ((gone >> b) & 1) sm.push_back(uni[b]);
      return contract(ins, sm);
    };
    return run(full);
  };
  for (int pi = 0; pi < ne; ++pi) {
    if (bucket[pi].empty()) continue;
    std::vector<int> inputs = bucket[pi];
    bucket[pi].clear();
    std::vector<int> uni;
    for (int id : inputs)
      for (int v : T[id].vars) uni.push_back(v);
    std::sort(uni.begin(), uni.end(), by_pos);
    uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
    int k = 1;
    // fuse the next variables of the union while every tensor holding them is
    // already in the product and brings no new variable
    while (k < max_fuse && k < (int)uni.size()) {
      int u = uni[k];
      int pu = pos[u];
      if (pu >= ne) break;
      // a wide bucket keeps at least 2^9 output entries per bitstring: the
      // resident kernels give each bitstring 256 threads, and an output
      // smaller than that makes lanes split the summed terms and reduce
      // across lanes (the rest is summed by the next, small, step)
      if ((int)uni.size() > 10 && (int)uni.size() - (k + 1) < 9) break;
      int in_inputs = 0;
      for (int id : inputs)
        if (std::find(T[id].vars.begin(), T[id].vars.end(), u) != T[id].vars.end()) ++in_inputs;
      if (live[u] != in_inputs + (int)bucket[pu].size()) break;
      bool subset = true;
      for (int id : bucket[pu])
        for (int v : T[id].vars)
          if (std::find(uni.begin(), uni.end(), v) == uni.end()) subset = false;
      if (!subset) break;
      for (int id : bucket[pu]) inputs.push_back(id);
      bucket[pu].clear();
      ++k;
    }
    shrink(inputs);
    const int oid = contract_tree(inputs, uni, k);
    place(oid);
  }
  // final product over the remaining tensors (scalars per batch entry, or
  // the tensor over the open outputs)
  if (finals.empty()) {
    set_error("internal: no final tensor");
  }
  std::vector<int> fin = finals;
  if (fin.size() == 1 && T[fin[0]].leaf < 0) {
    R.final_tensor = fin[0];
  } else {
    shrink(fin);
    int oid = emit(fin, {});
    R.final_tensor = oid;
  }
  R.final_tensors = finals;
  R.arena_peak = arena.peak;
  if (want_steps) {
    // bucket elimination is a tree: every tensor but the final one feeds
    // exactly one step
    std::vector<int> uses(T.size(), 0);
    for (const StepRec &st : R.steps)
      for (int id : st.inputs) uses[id]++;
    for (size_t id = 0; id < T.size(); ++id)
      if ((int)id != R.final_tensor && uses[id] != 1) {
        R.tree_error = (int)id;
        break;
      }
  }
  return R;
}

static int64_t pow2(int r) { return (int64_t)1 << r; }

// Table of model factor fi (inputs substituted by 0) on `scope`, optionally
// with the RXY table replaced by its derivative (which = 0: theta, 1: phi).
static std::vector<cd> member_table(const Model &m, int fi, const std::vector<int> &scope,
                                    int deriv_which) {
  const MFactor &f = m.factors[fi];
  cd t[4];
  for (int i = 0; i < 4; ++i) t[i] = f.t[i];
  if (deriv_which >= 0) {
    const qgm_gate &g = m.gates[f.gate];
    const cd I(0.0, 1.0);
    const double c = std::cos(g.theta / 2), sn = std::sin(g.theta / 2);
    if (deriv_which == 0) {  // d/dtheta of [[c, -i e^{-i phi} s], [-i e^{i phi} s, c]]
      t[0] = -0.5 * sn;
      t[1] = -I * std::exp(-I * g.phi) * (0.5 * c);
      t[2] = -I * std::exp(I * g.phi) * (0.5 * c);
      t[3] = -0.5 * sn;
    } else {  // d/dphi
      t[0] = 0.0;
      t[1] = -std::exp(-I * g.phi) * sn;
      t[2] = std::exp(I * g.phi) * sn;
      t[3] = 0.0;
    }
  }
  std::vector<char> is_in(m.n_vars, 0);
  for (int v : m.inputs) is_in[v] = 1;
  std::vector<int> keep;
  for (int a = 0; a < f.nv; ++a)
    if (!is_in[f.v[a]]) keep.push_back(a);
  std::vector<int> sc;
  for (int a : keep) sc.push_back(f.v[a]);
  std::vector<cd> tab((size_t)1 << keep.size());
  for (size_t i = 0; i < tab.size(); ++i) {
    int full = 0;
    for (size_t b = 0; b < keep.size(); ++b)
      if ((i >> (keep.size() - 1 - b)) & 1) full |= 1 << (f.nv - 1 - keep[b]);
    tab[i] = t[full];
  }
  return expand_table(sc, tab, scope);
}

// Index map of an operand whose variables `opvars` (most significant first)
// are a subset of the union `uni` (most significant first), as runs of
// contiguous union bits landing on contiguous operand bits.
static bool make_runs(const std::vector<int> &uni, const std::vector<int> &opvars, InDesc &in) {
  const int U = (int)uni.size(), R = (int)opvars.size();
  std::vector<int> vpos(U, -1);
  for (int b = 0; b < U; ++b) {
    const int v = uni[U - 1 - b];
    for (int a = 0; a < R; ++a)
      if (opvars[a] == v) vpos[b] = R - 1 - a;
  }
  int nr = 0, b = 0;
  while (b < U) {
    if (vpos[b] < 0) {
      ++b;
      continue;
    }
    const int st = b;
    ++b;
    while (b < U && vpos[b] == vpos[b - 1] + 1) ++b;
    if (nr >= MAXRUN) return false;
    in.src[nr] = (uint8_t)st;
    in.len[nr] = (uint8_t)(b - st);
    in.dst[nr] = (uint8_t)vpos[st];
    ++nr;
  }
  in.nruns = nr;
  return true;
}

// Offline placement of tensors whose lifetimes [born, dies] (dependency
// levels, inclusive) are known: largest first, each at the lowest 16-byte
// aligned offset not used by an already placed tensor of overlapping
// lifetime.  Returns the peak byte extent.
static int64_t pack_lifetimes(const std::vector<int64_t> &size, const std::vector<int> &born,
                              const std::vector<int> &dies, std::vector<int64_t> &off) {
  const int n = (int)size.size();
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return size[a] > size[b]; });
  off.assign(n, -1);
  std::vector<int> placed;
  int64_t peak = 0;
  for (int t : idx) {
    if (size[t] <= 0) continue;
    const int64_t sz = (size[t] + 15) & ~int64_t(15);
    std::vector<std::pair<int64_t, int64_t>> busy;  // [start, end) of conflicting tensors
    for (int u : placed)
      if (!(dies[u] < born[t] || dies[t] < born[u])) busy.push_back({off[u], off[u] + ((size[u] + 15) & ~int64_t(15))});
    std::sort(busy.begin(), busy.end());
    int64_t cand = 0;
    for (auto &b : busy) {
      if (b.first >= cand + sz) break;
      cand = std::max(cand, b.second);
    }
    off[t] = cand;
    peak = std::max(peak, cand + sz);
    placed.push_back(t);
  }
  return peak;
}

// Shared-memory layouts of the resident executor for chunks of Bc batch
// entries.  Steps are grouped into dependency levels (a step's level is one
// more than the highest level among the steps producing its inputs); the
// steps of a level are independent, run concurrently on disjoint warp groups
// and are followed by one block barrier.  The smem arena holds the leaves and
// intermediates with level-granular liveness (a level's outputs are placed
// before any of its inputs are released).
static void build_resident(qgm_plan *p) {
  p->resident.clear();
  if (p->output_mode != QGM_OUT_BATCH || !p->slice_vars.empty() || p->open_in_batch) return;
  const SimResult &S = p->sim;
  const int nl = (int)p->leaves.size();
  const int ns = (int)S.steps.size();
  // dependency levels
  std::vector<int> producer(S.tensors.size(), -1), level(ns, 0);
  int n_levels = 0;
  for (int si = 0; si < ns; ++si) {
    int l = 0;
    for (int id : S.steps[si].inputs)
      if (producer[id] >= 0) l = std::max(l, level[producer[id]] + 1);
    level[si] = l;
    producer[S.steps[si].out] = si;
    n_levels = std::max(n_levels, l + 1);
  }
  std::vector<int> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return level[a] < level[b]; });
  const int64_t meta_bytes = ((int64_t)p->n_meta * 8 + 15) & ~int64_t(15);
  // lifetimes in levels: leaves from the start, outputs from their level,
  // each until the level of its one consumer (the final tensor to the end)
  std::vector<int> born(S.tensors.size(), -1), dies(S.tensors.size(), n_levels);
  for (int si = 0; si < ns; ++si) {
    born[S.steps[si].out] = level[si];
    for (int id : S.steps[si].inputs) dies[id] = level[si];
  }
  // an output without a batch axis read by a batched step may be staged
  // before the first level (from the once-per-call part): live from the start
  for (int si = 0; si < ns; ++si)
    for (int id : S.steps[si].inputs)
      if (S.steps[si].batched && id >= nl && !S.tensors[id].batched) born[id] = -1;
  for (int Bc : {1, 2, 4, 8}) {
    ResidentLayout L;
    L.chunk = Bc;
    auto bytes_of = [&](const SymTensor &t) {
      return pow2((int)t.vars.size()) * (t.batched ? Bc : 1) * 8;
    };
    std::vector<int64_t> tsize(S.tensors.size()), where;
    for (size_t t = 0; t < S.tensors.size(); ++t) tsize[t] = bytes_of(S.tensors[t]);
    const int64_t arena_peak = pack_lifetimes(tsize, born, dies, where);
    std::vector<int64_t> soff = where;
    bool ok = true;
    for (int li = 0; li < nl; ++li) {
      const bool bt = S.tensors[li].batched;
      L.leaves.push_back({li, (int32_t)(meta_bytes + soff[li]), bt ? 1 : 0, 0});
      const LeafDesc &d = p->leafdesc[li];
      if (d.n_out > 2 || d.n_slice > 0) ok = false;
      for (int r = 0; r < (1 << d.n_int); ++r) {
        RJob j{};
        j.src = (int32_t)((d.base_off / 8) + ((int64_t)r << d.n_out));
        j.dst = (int32_t)(meta_bytes + soff[li] + (int64_t)r * (bt ? Bc : 1) * 8);
        j.n_out = (uint8_t)d.n_out;
        j.q0 = (uint8_t)(d.n_out > 0 ? d.out_qubit[0] : 0);
        j.q1 = (uint8_t)(d.n_out > 1 ? d.out_qubit[1] : 0);
        j.batched = bt ? 1 : 0;
        L.jobs.push_back(j);
      }
    }
    for (int lv = 0, pos = 0; lv < n_levels && ok; ++lv) {
      int end = pos;
      while (end < ns && level[order[end]] == lv) ++end;
      // warp groups: each step gets nw warps; longest steps first onto the
      // least-loaded contiguous warp range
      struct Job { int q, nw, lg; double cost; };
      std::vector<Job> jobs;
      for (int q = pos; q < end; ++q) {
        const StepDesc &d = p->steps[order[q]];
        const int64_t items = (int64_t)(1 << d.w_out) * (d.batched_out ? Bc : 1);
        const int64_t terms = (int64_t)1 << d.k;
        int nw = (int)std::min<int64_t>(RES_WARPS, std::max<int64_t>(1, (items * terms + 511) / 512));
        int lg = 0;
        const int Bco = d.batched_out ? Bc : 1;
        // more lanes per entry while entries are few, keeping a thread's
        // batch entry fixed (its item stride (32 nw) >> lg stays >= Bco)
        while (lg < 5 && lg < d.k && (items << (lg + 1)) <= 32 * nw && ((32 * nw) >> (lg + 1)) >= Bco) ++lg;
        const int64_t per_thread = ((items << lg) + 32 * nw - 1) / (32 * nw);
        jobs.push_back({q, nw, lg, (double)per_thread * (double)(terms >> lg) * d.m + 40.0});
      }
      std::stable_sort(jobs.begin(), jobs.end(), [](const Job &a, const Job &b) { return a.cost > b.cost; });
      double load[RES_WARPS] = {0};
      std::vector<int> w0_of(end - pos);
      for (const Job &j : jobs) {
        int best = 0;
        double bl = 1e300;
        for (int w = 0; w + j.nw <= RES_WARPS; ++w) {
          double mx = 0;
          for (int u = w; u < w + j.nw; ++u) mx = std::max(mx, load[u]);
          if (mx < bl) {
            bl = mx;
            best = w;
          }
        }
        for (int u = best; u < best + j.nw; ++u) load[u] = bl + j.cost;
        w0_of[j.q - pos] = best | (j.nw << 4) | (j.lg << 8);
      }
      for (int q = pos; q < end; ++q) {
        const int si = order[q];
        const StepRec &st = S.steps[si];
        const StepDesc &d = p->steps[si];
        const SymTensor &ot = S.tensors[st.out];
        RStep r{};
        r.m = d.m;
        r.k = d.k;
        r.w_out = d.w_out;
        r.batched_out = d.batched_out;
        r.out_soff = (int32_t)(meta_bytes + soff[st.out]);
        r.out_meta = ot.meta;
        r.sched = w0_of[q - pos] | (q == end - 1 ? SCHED_LAST : 0);
        for (int i = 0; i < d.m && ok; ++i) {
          const int id = st.inputs[i];
          const SymTensor &it = S.tensors[id];
          RIn &in = r.in[i];
          in.batched = it.batched ? 1 : 0;
          in.meta = it.leaf < 0 ? it.meta : -1;
          in.soff = (int32_t)(meta_bytes + where[id]);
          const int U = (int)st.uni.size();
          if (U > 32 || d.w_out > 16) {
            ok = false;
            break;
          }
          // value (element offset) of union bit b in this input, or 0
          std::vector<int64_t> v(U, 0);
          for (int qq = 0; qq < d.in[i].nruns; ++qq)
            for (int l = 0; l < d.in[i].len[qq]; ++l) v[d.in[i].src[qq] + l] = (int64_t)1 << (d.in[i].dst[qq] + l);
          const int bsh = it.batched ? (int)std::log2(Bc) : 0;
          const int64_t unit = (int64_t)8 << bsh;
          const int sched_lg = (w0_of[q - pos] >> 8) & 15, sched_nw = (w0_of[q - pos] >> 4) & 15;
          const int Bco = d.batched_out ? Bc : 1;
          const int sit = (32 * sched_nw) >> sched_lg;
          int r0 = 0;
          while ((1 << (r0 + 1)) <= sit / Bco) ++r0;
          in.nlow = std::min(r0, d.w_out);
          for (int t = 0; t < 16; ++t) {
            int64_t val = 0;
            if (t < d.w_out - r0) {
              val = v[r0 + t];
              for (int b = 0; b < t; ++b) val -= v[r0 + b];
            }
            in.rinc[t] = (int32_t)(val * unit);
          }
          for (int t = 0; t < 8; ++t) {
            int64_t val = 0;
            if (t < d.k - sched_lg) {
              val = v[d.w_out + sched_lg + t];
              for (int b = 0; b < t; ++b) val -= v[d.w_out + sched_lg + b];
            }
            in.tinc[t] = (int32_t)(val * unit);
          }
          for (int b = 0; b < 8; ++b) {
            in.lrow[b] = b < in.nlow ? (int32_t)(v[b] * unit) : 0;
            in.lterm[b] = b < sched_lg ? (int32_t)(v[d.w_out + b] * unit) : 0;
          }
        }
        r.bytes = (int32_t)(offsetof(RStep, in) + d.m * sizeof(RIn));
        L.steps.push_back(r);
        L.src_step.push_back(si);
        L.level.push_back(lv);
      }
      pos = end;
    }
    if (!ok) break;  // an index map too fragmented for the resident kernel
    L.final_soff = (int)(meta_bytes + where[S.final_tensor]);
    L.final_meta = S.tensors[S.final_tensor].meta;
    L.smem_bytes = meta_bytes + arena_peak;
    // per-warp work lists, then move the arena behind them in shared memory
    L.n_levels = n_levels;
    {
      std::vector<std::vector<uint32_t>> per(RES_WARPS);
      for (size_t q = 0; q < L.steps.size(); ++q) {
        const RStep &r = L.steps[q];
        const int w0 = r.sched & 15, nw = (r.sched >> 4) & 15;
        const uint32_t words = (uint32_t)(r.bytes / 4);
        const uint32_t lvl = (uint32_t)level[order[q]];
        if (q >= 4096 || lvl >= 1024 || words >= 1024) ok = false;
        for (int w = w0; w < w0 + nw; ++w) per[w].push_back((uint32_t)q | (lvl << 12) | (words << 22));
      }
      L.wstart[0] = 0;
      for (int w = 0; w < RES_WARPS; ++w) {
        L.wlist.insert(L.wlist.end(), per[w].begin(), per[w].end());
        L.wstart[w + 1] = (int32_t)L.wlist.size();
      }
      const int64_t shift = ((int64_t)L.wlist.size() * 4 + 15) & ~int64_t(15);
      L.wlist_soff = (int)meta_bytes;
      for (RStep &r : L.steps) {
        r.out_soff += (int32_t)shift;
        for (int i = 0; i < r.m; ++i) r.in[i].soff += (int32_t)shift;
      }
      for (RJob &j : L.jobs) j.dst += (int32_t)shift;
      for (RLeaf &lf : L.leaves) lf.soff += (int32_t)shift;
      L.final_soff += (int)shift;
      L.smem_bytes += shift;
    }
    if (!ok) break;
    if (L.smem_bytes > 200 * 1024) break;  // larger chunks only grow
    // leaf rows read from the bitstrings first (the compiled kernel stages
    // only those one by one; the others come with its shared-memory image)
    std::stable_partition(L.jobs.begin(), L.jobs.end(), [](const RJob &j) { return j.batched != 0; });
    p->resident.push_back(L);
  }
  {
    int64_t image = 0;
    for (const ResidentLayout &L : p->resident) image = std::max(image, compiled_smem(L));
    if (image > 0) {
      p->off_image = p->ws_bytes - 256;
      p->ws_bytes += (image + 255) & ~int64_t(255);
    }
  }
  // bitstring-independent outputs read by batched steps (the same tensors and
  // pre-region places in every layout)
  std::vector<int> consumer(S.tensors.size(), -1);
  for (int si = 0; si < ns; ++si)
    for (int id : S.steps[si].inputs) consumer[id] = si;
  const bool final_batched = S.tensors[S.final_tensor].batched;
  for (ResidentLayout &L : p->resident) {
    int64_t goff = 0;
    for (size_t q = 0; q < L.steps.size(); ++q) {
      const StepRec &st = S.steps[L.src_step[q]];
      if (st.batched) continue;
      const int c = consumer[st.out];
      if (c < 0 || !S.steps[c].batched) continue;
      const int64_t n = pow2((int)S.tensors[st.out].vars.size());
      L.pre.push_back({L.steps[q].out_soff, L.steps[q].out_meta, (int32_t)n, (int32_t)goff});
      goff += (n + 1) & ~int64_t(1);
    }
    L.split_pre = final_batched && !L.pre.empty();
    if (L.split_pre) {
      const int64_t meta_b = ((int64_t)L.pre.size() * 8 + 15) & ~int64_t(15);
      p->pre_data = meta_b / 8;
      const int64_t need = meta_b + goff * 8;
      if (p->off_pre == 0) {
        p->off_pre = p->ws_bytes - 256;
        p->ws_bytes += (need + 255) & ~int64_t(255);
      }
    }
  }
}

// Numeric contents of the base tables (complex64): each leaf's table laid
// out over (internal | slice | output variables), and, with gradients, the
// derivative tables of the leaves holding an RXY gate -- d(leaf)/dp = product
// of the other members x d(RXY)/dp, for p = theta and phi.
static void fill_tables(qgm_plan *p) {
  const Model &m = p->model;
  for (size_t li = 0; li < p->leaves.size(); ++li) {
    const LeafFactor &L = p->leaves[li];
    const std::vector<int> &layout = p->leaf_layout[li];
    std::vector<cd> tab = expand_table(L.scope, L.table, layout);
    for (size_t i = 0; i < tab.size(); ++i) {
      p->base_tables[p->base_at[li] + 2 * i] = (float)tab[i].real();
      p->base_tables[p->base_at[li] + 2 * i + 1] = (float)tab[i].imag();
    }
    if (p->grad && p->rxy_member[li] >= 0) {
      for (int which = 0; which < 2; ++which) {
        std::vector<cd> dt(tab.size(), 1.0);
        for (int fi : L.members) {
          std::vector<cd> mt = member_table(m, fi, layout, fi == p->rxy_member[li] ? which : -1);
          for (size_t i = 0; i < dt.size(); ++i) dt[i] *= mt[i];
        }
        const int64_t at = p->dbase_at[li] + 2 * which * (int64_t)tab.size();
        for (size_t i = 0; i < dt.size(); ++i) {
          p->base_tables[at + 2 * i] = (float)dt[i].real();
          p->base_tables[at + 2 * i + 1] = (float)dt[i].imag();
        }
      }
    }
  }
}

// New angles for the RXY gates of the plan's circuit (params: theta_p at 2p,
// phi_p at 2p+1, the order of qgm_circuit_param_gates): the gate tables,
// the merged leaf tables and the constant are recomputed on the host; the
// variable structure -- and so the order, the steps and the layout -- does
// not depend on the angles.
int plan_set_params(qgm_plan *p, const double *params) {
  Model &m = p->model;
  for (size_t q = 0; q < m.param_factor.size(); ++q) {
    MFactor &f = m.factors[m.param_factor[q]];
    qgm_gate &g = m.gates[f.gate];
    g.theta = params[2 * q];
    g.phi = params[2 * q + 1];
    gate_table(g, f.t, &f.half_pow);
  }
  std::vector<LeafFactor> leaves;
  cd constant;
  int hp = 0;
  reduce_factors(m, leaves, constant, hp);
  if (leaves.size() != p->leaves.size() || hp != p->half_pow_total) {
    set_error("qgm_plan_set_params: the leaf structure changed");
    return QGM_ERR_ARG;
  }
  for (size_t li = 0; li < leaves.size(); ++li) {
    if (leaves[li].scope != p->leaves[li].scope || leaves[li].members != p->leaves[li].members) {
      set_error("qgm_plan_set_params: the leaf structure changed");
      return QGM_ERR_ARG;
    }
    p->leaves[li].table = leaves[li].table;
  }
  p->constant = constant;
  fill_tables(p);
  return QGM_OK;
}

int build_plan(const Model &m, const qgm_plan_opts &o, qgm_plan *p) {
  p->model = m;
  p->opts = o;
  p->opts.order = nullptr;
  p->opts.keep_vars = nullptr;
  p->output_mode = o.output_mode;
  if (o.output_mode != QGM_OUT_BATCH && o.output_mode != QGM_OUT_OPEN) {
    set_error("qgm_plan_order: bad output_mode %d", o.output_mode);
    return QGM_ERR_ARG;
  }
  if (o.output_mode == QGM_OUT_BATCH) {
    if (o.batch < 1 || o.batch > (1 << 24)) {
      set_error("qgm_plan_order: batch %lld out of [1, 2^24]", (long long)o.batch);
      return QGM_ERR_ARG;
    }
    p->batch = o.batch;
    p->Bp = (int32_t)((o.batch + 3) / 4 * 4);
  } else {
    if (m.n > 30) {
      set_error("qgm_plan_order: open outputs need n <= 30 (got %d)", m.n);
      return QGM_ERR_ARG;
    }
    p->batch = 1;
    p->Bp = 1;
  }
  const int max_fuse = o.max_fuse > 0 ? std::min(o.max_fuse, 16) : 8;
  p->gemm_ok = o.no_gemm == 0;
  p->gemm_tc = o.gemm_precision >= 0;
  p->tc_planes = o.gemm_precision == 1 ? 6 : 4;
  if (o.gemm_precision < -1 || o.gemm_precision > 2) {
    set_error("qgm_plan_order: bad gemm_precision %d", o.gemm_precision);
    return QGM_ERR_ARG;
  }
  p->trees_ok = o.trees > 0;
  p->nest_ok = true;
  const int64_t budget = o.mem_budget_bytes > 0 ? o.mem_budget_bytes : (int64_t)64 << 30;

  reduce_factors(m, p->leaves, p->constant, p->half_pow_total);
  p->var_role.assign(m.n_vars, 0);
  for (int v : m.inputs) p->var_role[v] = 1;
  p->open_vars.clear();
  if (o.output_mode == QGM_OUT_BATCH && m.n < 64 && (o.open_mask >> m.n) != 0) {
    set_error("qgm_plan_order: open_mask names qubits beyond n = %d", m.n);
    return QGM_ERR_ARG;
  }
  p->open_in_batch = 0;
  for (int q = m.n - 1; q >= 0; --q) {
    int v = m.outputs[q];
    if (p->var_role[v] == 1) continue;  // qubit without gates: output = input
    const bool open_here = o.output_mode == QGM_OUT_BATCH && ((o.open_mask >> q) & 1);
    if (o.output_mode == QGM_OUT_BATCH && !open_here) p->var_role[v] = 2;
    else {
      p->open_in_batch += open_here;
      p->var_role[v] = 3;
      p->open_vars.push_back(v);
    }
  }
  for (int q = 0; q < m.n; ++q)
    if (p->var_role[m.outputs[q]] == 1) {
      set_error("qgm_plan_order: qubit %d has no non-diagonal gate (every qubit needs one)", q);
      return QGM_ERR_ARG;
    }
  // variables kept open on request (a batch plan): never eliminated, like
  // open outputs; keep_vars[j] is bit j of the low part of the entry index
  if (o.n_keep < 0 || (o.n_keep > 0 && (!o.keep_vars || o.output_mode != QGM_OUT_BATCH))) {
    set_error("qgm_plan_order: keep_vars needs a batch plan and a list");
    return QGM_ERR_ARG;
  }
  for (int j = o.n_keep - 1; j >= 0; --j) {
    const int v = o.keep_vars[j];
    if (v < 0 || v >= m.n_vars || p->var_role[v] == 1 || p->var_role[v] == 3) {
      set_error("qgm_plan_order: keep_vars holds %d (an input, an open output, repeated or unknown)", v);
      return QGM_ERR_ARG;
    }
    p->var_role[v] = 3;
    p->open_vars.push_back(v);
    p->open_in_batch += 1;
  }
  std::vector<char> in_graph(m.n_vars, 0), elim(m.n_vars, 0), keep(m.n_vars, 0);
  for (int v = 0; v < m.n_vars; ++v) {
    in_graph[v] = p->var_role[v] == 0 || p->var_role[v] == 3;
    elim[v] = p->var_role[v] == 0;
    keep[v] = p->var_role[v] == 3;
  }
  Graph g = make_graph(p, in_graph);

  std::vector<std::pair<int, std::vector<int>>> cands;
  int kind = o.order_kind;
  if (kind == QGM_ORDER_GIVEN) {
    if (!o.order || o.n_order < 0) {
      set_error("qgm_plan_order: QGM_ORDER_GIVEN without an order");
      return QGM_ERR_ARG;
    }
    std::vector<int> given(o.order, o.order + o.n_order);
    std::vector<char> seen(m.n_vars, 0);
    for (int v : given) {
      if (v < 0 || v >= m.n_vars || !elim[v] || seen[v]) {
        set_error("qgm_plan_order: given order holds %d, not a free variable (or repeated)", v);
        return QGM_ERR_ARG;
      }
      seen[v] = 1;
    }
    for (int v = 0; v < m.n_vars; ++v)
      if (elim[v] && !seen[v]) {
        set_error("qgm_plan_order: given order misses variable %d", v);
        return QGM_ERR_ARG;
      }
    cands.push_back({QGM_ORDER_GIVEN, given});
  } else {
    if (kind < 0 || kind > QGM_ORDER_VERTICAL_T) {
      set_error("qgm_plan_order: bad order_kind %d", kind);
      return QGM_ERR_ARG;
    }
    if (kind == QGM_ORDER_AUTO || kind == QGM_ORDER_MINFILL)
      cands.push_back({QGM_ORDER_MINFILL, order_minfill(g, keep)});
    if (kind == QGM_ORDER_AUTO || kind == QGM_ORDER_VERTICAL)
      cands.push_back({QGM_ORDER_VERTICAL, order_vertical(p, elim, false)});
    if (kind == QGM_ORDER_AUTO || kind == QGM_ORDER_VERTICAL_T)
      cands.push_back({QGM_ORDER_VERTICAL_T, order_vertical(p, elim, true)});
  }
  // slice each candidate until its live set fits, keep the cheapest
  double best_cost = -1;
  for (auto &c : cands) {
    std::vector<char> sliced(m.n_vars, 0);
    std::vector<int> svars;
    SimResult r = simulate(p, c.second, sliced, max_fuse, false);
    while (r.arena_peak > budget && svars.size() < 40) {
      // the variable in the most cliques of the largest size along the
      // order, on the graph without the variables sliced so far (ties:
      // smallest id)
      std::vector<char> ig = in_graph;
      for (int v = 0; v < m.n_vars; ++v)
        if (sliced[v]) ig[v] = 0;
      Graph gs = make_graph(p, ig);
      std::vector<std::vector<int>> cl;
      size_t mx = 0;
      for (int v : c.second) {
        if (sliced[v]) continue;
        std::vector<int> q = gs.nbrs(v);
        q.push_back(v);
        mx = std::max(mx, q.size());
        cl.push_back(std::move(q));
        gs.eliminate(v);
      }
      std::vector<int> cnt(m.n_vars, 0);
      for (const auto &q : cl)
        if (q.size() == mx)
          for (int v : q)
            if (p->var_role[v] == 0) cnt[v]++;
      int bv = -1;
      for (int v = 0; v < m.n_vars; ++v)
        if (cnt[v] > 0 && (bv < 0 || cnt[v] > cnt[bv])) bv = v;
      if (bv < 0) break;
      sliced[bv] = 1;
      svars.push_back(bv);
      r = simulate(p, c.second, sliced, max_fuse, false);
    }
    if (r.arena_peak > budget) continue;
    double cost = r.bytes * (double)pow2((int)svars.size());
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      p->order_kind = c.first;
      p->order = c.second;
      p->slice_vars = svars;
    }
  }
  if (best_cost < 0) {
    set_error("qgm_plan_order: no order fits the memory budget of %lld bytes even sliced",
              (long long)budget);
    return QGM_ERR_OOM;
  }
  std::vector<char> sliced(m.n_vars, 0);
  for (int v : p->slice_vars) {
    sliced[v] = 1;
    p->var_role[v] = 4;
  }
  p->sim = simulate(p, p->order, sliced, max_fuse, true);
  SimResult &S = p->sim;
  if (S.tree_error >= 0) {
    set_error("internal: tensor %d of the elimination is consumed other than once", S.tree_error);
    return QGM_ERR_ARG;
  }
  // induced width along the order on the graph without the sliced variables
  {
    std::vector<char> ig = in_graph;
    for (int v : p->slice_vars) ig[v] = 0;
    Graph g2 = make_graph(p, ig);
    int w = 0;
    for (int v : p->order)
      if (!sliced[v]) w = std::max(w, g2.eliminate(v));
    S.max_clique = w;
  }
  p->pos.assign(m.n_vars, -1);
  {
    int i = 0;
    for (int v : p->order)
      if (!sliced[v]) p->pos[v] = i++;
    for (size_t j = 0; j < p->open_vars.size(); ++j) p->pos[p->open_vars[j]] = i + (int)j;
  }

  // ---------------------------------------------------- device layout
  const int64_t Bp = p->Bp;
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    int64_t o2 = off;
    off += (bytes + 255) & ~int64_t(255);
    return o2;
  };
  int n_meta = 0;
  for (const SymTensor &t : S.tensors)
    if (t.leaf < 0) n_meta = std::max(n_meta, t.meta + 1);
  p->n_meta = n_meta;
  p->n_meta_fwd = n_meta;
  p->grad = o.gradients != 0;
  if (p->grad && (o.output_mode != QGM_OUT_BATCH || p->open_in_batch)) {
    set_error("qgm_plan_order: gradients need a batch plan without open outputs");
    return QGM_ERR_ARG;
  }
  // with gradients: one more slot per adjoint (at most one per tensor) + seed
  const int meta_slots = p->grad ? (int)(n_meta + S.tensors.size() + 2) : n_meta;
  p->off_header = take(256);
  p->off_meta = take((int64_t)std::max(meta_slots, 1) * 8);
  p->off_leafdesc = take((int64_t)std::max<size_t>(p->leaves.size(), 1) * sizeof(LeafDesc));
  // base tables: (internal vars by position | slice vars | output vars by qubit)
  p->base_tables.clear();
  p->leafdesc.clear();
  std::vector<int64_t> leaf_built_off(p->leaves.size(), -1);
  int64_t base_floats = 0;
  std::vector<int64_t> base_at(p->leaves.size());
  for (size_t li = 0; li < p->leaves.size(); ++li) {
    base_at[li] = base_floats;
    base_floats += 2 * (int64_t)p->leaves[li].table.size();
    base_floats = (base_floats + 3) & ~int64_t(3);
  }
  // derivative tables (theta, phi) of the leaves that hold an RXY gate
  std::vector<int> rxy_member(p->leaves.size(), -1);
  std::vector<int64_t> dbase_at(p->leaves.size(), -1);
  if (p->grad) {
    for (size_t li = 0; li < p->leaves.size(); ++li)
      for (int fi : p->leaves[li].members)
        if (m.gates[m.factors[fi].gate].kind == QGM_GATE_RXY) rxy_member[li] = fi;
    for (size_t li = 0; li < p->leaves.size(); ++li)
      if (rxy_member[li] >= 0) {
        dbase_at[li] = base_floats;
        base_floats += 4 * (int64_t)p->leaves[li].table.size();
        base_floats = (base_floats + 3) & ~int64_t(3);
      }
  }
  p->off_base = take(base_floats * 4);
  p->base_tables.assign(base_floats, 0.f);
  p->leaf_layout.clear();
  p->base_at = base_at;
  p->dbase_at = dbase_at;
  p->rxy_member = rxy_member;
  int64_t leaf_bytes = 0;
  for (size_t li = 0; li < p->leaves.size(); ++li) {
    const LeafFactor &L = p->leaves[li];
    const SymTensor &t = S.tensors[li];
    std::vector<int> intv = t.vars, slv, outv;
    for (int v : L.scope) {
      if (p->var_role[v] == 4) slv.push_back(v);
      if (p->var_role[v] == 2) outv.push_back(v);
    }
    std::sort(slv.begin(), slv.end(), [&](int a, int b) {
      return std::find(p->slice_vars.begin(), p->slice_vars.end(), a) <
             std::find(p->slice_vars.begin(), p->slice_vars.end(), b);
    });
    std::sort(outv.begin(), outv.end(),
              [&](int a, int b) { return m.var_qubit[a] < m.var_qubit[b]; });
    std::vector<int> layout = intv;
    layout.insert(layout.end(), slv.begin(), slv.end());
    layout.insert(layout.end(), outv.begin(), outv.end());
    if ((int)layout.size() > MAXLEAFV || layout.size() != L.scope.size()) {
      set_error("internal: leaf %zu has %zu variables", li, layout.size());
      return QGM_ERR_ARG;
    }
    p->leaf_layout.push_back(layout);
    LeafDesc d{};
    d.base_off = p->off_base + base_at[li] * 4;
    d.n_int = (int)intv.size();
    d.n_slice = (int)slv.size();
    d.n_out = (int)outv.size();
    d.batched = t.batched ? 1 : 0;
    for (size_t a = 0; a < slv.size(); ++a)
      d.slice_bit[a] = (int)(std::find(p->slice_vars.begin(), p->slice_vars.end(), slv[a]) -
                             p->slice_vars.begin());
    for (size_t a = 0; a < outv.size(); ++a) d.out_qubit[a] = m.var_qubit[outv[a]];
    d.out_off = leaf_bytes;  // relative, fixed below
    leaf_bytes += ((pow2(d.n_int) * (d.batched ? Bp : 1) * 8) + 255) & ~int64_t(255);
    p->leafdesc.push_back(d);
  }
  fill_tables(p);
  p->off_leaf = take(leaf_bytes);
  for (size_t li = 0; li < p->leafdesc.size(); ++li) {
    p->leafdesc[li].out_off += p->off_leaf;
    S.tensors[li].off = p->leafdesc[li].out_off;
  }
  p->off_bits = take(Bp * 8);
  const SymTensor &F = S.tensors[S.final_tensor];
  p->final_entries = pow2((int)F.vars.size());
  p->final_batched = F.batched ? 1 : 0;
  if (p->open_in_batch > 20) {
    set_error("qgm_plan_order: at most 20 open outputs in a batch plan");
    return QGM_ERR_ARG;
  }
  int64_t out_elems = o.output_mode == QGM_OUT_BATCH ? (Bp << p->open_in_batch) : p->final_entries;
  p->off_outstage = take(out_elems * 16);
  p->off_acc = take(out_elems * 16);
  {
    int64_t njobs = 0;
    for (size_t li = 0; li < p->leaves.size(); ++li)
      njobs += (int64_t)1 << (S.tensors[li].vars.size());
    p->off_rsteps = take((int64_t)(S.steps.size() + 1) * sizeof(RStep) +
                         (int64_t)(p->leaves.size() + 1) * sizeof(RLeaf) + (njobs + 1) * sizeof(RJob) +
                         ((int64_t)S.steps.size() * RES_WARPS + RES_WARPS + 8) * 4);
  }
  p->off_sdesc = take((int64_t)(S.steps.size() + 1) * (int64_t)sizeof(StepDesc));
  p->off_arena = take(0);
  for (SymTensor &t : S.tensors)
    if (t.leaf < 0) t.off += p->off_arena;
  p->ws_bytes = p->off_arena + ((S.arena_peak + 255) & ~int64_t(255)) + 256;
  p->final_off = F.off;
  p->final_meta = F.leaf < 0 ? F.meta : -1;

  // step descriptors
  p->steps.clear();
  p->gemms.clear();
  p->executor_pref = o.executor;
  for (const StepRec &s : S.steps) {
    StepDesc d{};
    d.gemm = -1;
    if (s.gemm) {
      // operand and output bit positions of each kind of variable
      const SymTensor &A = S.tensors[s.inputs[0]], &B = S.tensors[s.inputs[1]], &O = S.tensors[s.out];
      auto bitpos = [](const SymTensor &t, int v) {
        const int a = (int)(std::find(t.vars.begin(), t.vars.end(), v) - t.vars.begin());
        return a < (int)t.vars.size() ? (int)t.vars.size() - 1 - a : -1;
      };
      std::vector<int> mv, nv, kv, sv;
      for (size_t a = 0; a < s.uni.size(); ++a) {
        const int v = s.uni[a];
        const int pa = bitpos(A, v), pb = bitpos(B, v);
        if ((int)a < s.k) kv.push_back(v);
        else if (pa >= 0 && pb >= 0) sv.push_back(v);
        else if (pa >= 0) mv.push_back(v);
        else nv.push_back(v);
      }
      std::sort(mv.begin(), mv.end(), [&](int x, int y) { return bitpos(A, x) < bitpos(A, y); });
      std::sort(nv.begin(), nv.end(), [&](int x, int y) { return bitpos(B, x) < bitpos(B, y); });
      std::sort(kv.begin(), kv.end(), [&](int x, int y) { return bitpos(A, x) < bitpos(A, y); });
      std::sort(sv.begin(), sv.end(), [&](int x, int y) { return bitpos(O, x) < bitpos(O, y); });
      GemmDesc g{};
      g.a_off = A.off;
      g.b_off = B.off;
      g.o_off = O.off;
      g.a_meta = A.leaf < 0 ? A.meta : -1;
      g.b_meta = B.leaf < 0 ? B.meta : -1;
      g.o_meta = O.meta;
      g.a_bat = A.batched;
      g.b_bat = B.batched;
      g.o_bat = O.batched;
      g.nm = (int)mv.size();
      g.nn = (int)nv.size();
      g.nk = (int)kv.size();
      g.ns = (int)sv.size();
      if (g.nm >= GMAXB || g.nn >= GMAXB || g.nk >= GMAXB || g.ns >= GMAXB || g.ns > 15) {
        set_error("internal: GEMM step too wide");
        return QGM_ERR_ARG;
      }
      for (int b = 0; b < g.nm; ++b) { g.mA[b] = (uint8_t)bitpos(A, mv[b]); g.mO[b] = (uint8_t)bitpos(O, mv[b]); }
      for (int b = 0; b < g.nn; ++b) { g.nB[b] = (uint8_t)bitpos(B, nv[b]); g.nO[b] = (uint8_t)bitpos(O, nv[b]); }
      for (int b = 0; b < g.nk; ++b) { g.kA[b] = (uint8_t)bitpos(A, kv[b]); g.kB[b] = (uint8_t)bitpos(B, kv[b]); }
      for (int b = 0; b < g.ns; ++b) {
        g.sA[b] = (uint8_t)bitpos(A, sv[b]);
        g.sB[b] = (uint8_t)bitpos(B, sv[b]);
        g.sO[b] = (uint8_t)bitpos(O, sv[b]);
      }
      d.gemm = (int)p->gemms.size();
      p->gemms.push_back(g);
    }
    d.m = (int)s.inputs.size();
    d.k = s.k;
    const int U = (int)s.uni.size();
    d.w_out = U - s.k;
    const SymTensor &ot = S.tensors[s.out];
    d.batched_out = ot.batched ? 1 : 0;
    d.out_off = ot.off;
    d.out_meta = ot.meta;
    for (int i = 0; i < d.m; ++i) {
      const SymTensor &it = S.tensors[s.inputs[i]];
      InDesc &in = d.in[i];
      in.off = it.off;
      in.meta = it.leaf < 0 ? it.meta : -1;
      in.batched = it.batched ? 1 : 0;
      // union bit of var a is U-1-a; summed variables come first in the
      // union, so an input's bits may land out of order (general runs)
      if (!make_runs(s.uni, it.vars, in)) {
        set_error("internal: index map with more than %d runs", MAXRUN);
        return QGM_ERR_ARG;
      }
    }
    // register tile for large batched steps whose output has bits the
    // largest input lacks (those outputs reuse its loaded values)
    d.tile_t = 0;
    if (d.batched_out && d.gemm < 0) {
      int big = 0;
      for (int i = 1; i < d.m; ++i)
        if (S.tensors[s.inputs[i]].entries > S.tensors[s.inputs[big]].entries) big = i;
      const SymTensor &bt = S.tensors[s.inputs[big]];
      if (bt.batched && bt.entries * 8 >= ((int64_t)1 << 22)) {
        for (int b = 0; b < d.w_out && d.tile_t < 3; ++b) {
          const int v = s.uni[U - 1 - b];
          if (std::find(bt.vars.begin(), bt.vars.end(), v) == bt.vars.end()) d.tile_pos[d.tile_t++] = (uint8_t)b;
        }
        if (d.w_out - d.tile_t < 1) d.tile_t = 0;
        // inputs holding tile bits are reloaded for every tile entry: only
        // worth it when they are small next to the largest input
        for (int i = 0; i < d.m && d.tile_t > 0; ++i) {
          if (i == big) continue;
          const SymTensor &it = S.tensors[s.inputs[i]];
          bool holds = false;
          for (int q = 0; q < d.tile_t; ++q)
            holds |= std::find(it.vars.begin(), it.vars.end(), s.uni[U - 1 - d.tile_pos[q]]) != it.vars.end();
          if (holds && it.entries * 8 > bt.entries) d.tile_t = 0;
        }
      }
    }
    p->steps.push_back(d);
  }
  // batch-outer intermediates: the output of a tensor-core product per batch
  // entry whose only reader is another tensor-core step's operand split (each
  // entry's stores are then contiguous instead of 8 bytes in every 32-byte
  // sector); large tensors only, none in a gradient layout (its product-sum
  // kernels read batch-inner rows)
  if (p->gemm_tc && !p->grad) {
    std::vector<int> consumer(S.tensors.size(), -1);
    for (size_t si = 0; si < S.steps.size(); ++si)
      for (int id : S.steps[si].inputs) consumer[id] = (int)si;
    for (size_t si = 0; si < S.steps.size(); ++si) {
      const StepDesc &d = p->steps[si];
      if (d.gemm < 0) continue;
      GemmDesc &g = p->gemms[d.gemm];
      const TcCfg c = tc_config(g, (int)Bp, p->tc_planes);
      const int out = S.steps[si].out;
      if (!c.ok || !c.perbeta || S.tensors[out].entries < ((int64_t)1 << 24)) continue;
      const int cs = consumer[out];
      if (cs < 0 || p->steps[cs].gemm < 0) continue;
      GemmDesc &h = p->gemms[p->steps[cs].gemm];
      if (!tc_config(h, (int)Bp, p->tc_planes).ok) continue;
      if (h.a_off == g.o_off) h.a_bout = 1;
      else if (h.b_off == g.o_off) h.b_bout = 1;
      else continue;
      g.o_bout = 1;
    }
  }
  p->tune.assign(p->steps.size(), StepTune{});
  // runs of at least two consecutive small batch-free product-sum steps (at
  // most 2^12 outputs and 2^16 products each): a launch of their own would
  // cost more than the work
  p->plain_group.assign(p->steps.size(), 0);
  for (size_t s0 = 0; s0 < p->steps.size();) {
    auto small = [&](size_t s) {
      const StepDesc &d = p->steps[s];
      return d.gemm < 0 && !d.batched_out && d.w_out <= 12 && d.w_out + d.k <= 16;
    };
    size_t s1 = s0;
    while (s1 < p->steps.size() && small(s1)) ++s1;
    if (s1 - s0 >= 2) p->plain_group[s0] = (int32_t)(s1 - s0);
    s0 = s1 > s0 ? s1 : s0 + 1;
  }
  // the split operand planes of the largest tensor-core step, after the arena
  p->ws_fwd_bytes = p->ws_bytes;
  p->planes_bytes = 0;
  if (p->gemm_tc)
    for (const GemmDesc &g : p->gemms) {
      const TcCfg c = tc_config(g, (int)Bp, p->tc_planes);
      if (c.ok) p->planes_bytes = std::max(p->planes_bytes, c.bytesM + c.bytesN);
    }
  p->off_planes = p->ws_bytes - 256;
  p->ws_bytes = p->off_planes + p->planes_bytes + 256;
  build_resident(p);
  if (p->grad) {
    // ------------------------------------------- adjoint elimination layout
    // forward intermediates keep their own region (no reuse); adjoints too
    int64_t goff = p->ws_bytes - 256;
    auto gtake = [&](int64_t bytes) {
      int64_t o2 = goff;
      goff += (bytes + 255) & ~int64_t(255);
      return o2;
    };
    const int nt = (int)S.tensors.size();
    std::vector<int64_t> fwd_off(nt, -1);
    for (int t = 0; t < nt; ++t)
      fwd_off[t] = S.tensors[t].leaf >= 0 ? S.tensors[t].off : gtake(S.tensors[t].entries * 8);
    // which tensors lead to a parametrised leaf
    std::vector<char> need(nt, 0);
    for (size_t li = 0; li < p->leaves.size(); ++li) need[li] = rxy_member[li] >= 0;
    for (const StepRec &st : S.steps)
      for (int id : st.inputs) need[st.out] |= need[id];
    p->gfwd = p->steps;
    for (size_t si = 0; si < S.steps.size(); ++si) {
      StepDesc &d = p->gfwd[si];
      d.gemm = -1;
      d.tile_t = 0;
      d.out_off = fwd_off[S.steps[si].out];
      for (int i = 0; i < d.m; ++i) d.in[i].off = fwd_off[S.steps[si].inputs[i]];
    }
    const SymTensor &Fg = S.tensors[S.final_tensor];
    p->g_final_off = fwd_off[S.final_tensor];
    p->g_final_meta = Fg.leaf < 0 ? Fg.meta : -1;
    p->g_final_batched = Fg.batched ? 1 : 0;
    if (Fg.leaf >= 0 || !Fg.vars.empty() || !Fg.batched) {
      set_error("internal: gradient needs a batched rank-0 final tensor");
      return QGM_ERR_ARG;
    }
    // adjoints: the seed for the final tensor (ones), then one per needed input
    std::vector<int64_t> adj_off(nt, -1);
    std::vector<int> adj_meta(nt, -1);
    int next_meta = p->n_meta_fwd;
    adj_off[S.final_tensor] = gtake(Bp * 8);
    adj_meta[S.final_tensor] = next_meta++;
    p->g_seed_off = adj_off[S.final_tensor];
    p->g_seed_meta = adj_meta[S.final_tensor];
    p->gbwd.clear();
    for (int si = (int)S.steps.size() - 1; si >= 0; --si) {
      const StepRec &st = S.steps[si];
      if (!need[st.out] || adj_off[st.out] < 0) continue;
      const SymTensor &ot = S.tensors[st.out];
      for (size_t i = 0; i < st.inputs.size(); ++i) {
        const int id = st.inputs[i];
        if (!need[id]) continue;
        const SymTensor &it = S.tensors[id];
        // union: the variables summed here first, then the input's own
        std::vector<int> summed, uni;
        for (int v : st.uni)
          if (std::find(it.vars.begin(), it.vars.end(), v) == it.vars.end()) summed.push_back(v);
        uni = summed;
        uni.insert(uni.end(), it.vars.begin(), it.vars.end());
        StepDesc d{};
        d.gemm = -1;
        d.tile_t = 0;
        d.k = (int)summed.size();
        d.w_out = (int)it.vars.size();
        d.batched_out = 1;
        adj_off[id] = gtake(pow2(d.w_out) * Bp * 8);
        adj_meta[id] = next_meta++;
        d.out_off = adj_off[id];
        d.out_meta = adj_meta[id];
        int mm = 0;
        InDesc &a0 = d.in[mm++];
        a0.off = adj_off[st.out];
        a0.meta = adj_meta[st.out];
        a0.batched = 1;
        bool ok = make_runs(uni, ot.vars, a0);
        for (size_t k2 = 0; k2 < st.inputs.size() && ok; ++k2) {
          if (k2 == i) continue;
          const SymTensor &kt = S.tensors[st.inputs[k2]];
          InDesc &ik = d.in[mm++];
          ik.off = fwd_off[st.inputs[k2]];
          ik.meta = kt.leaf < 0 ? kt.meta : -1;
          ik.batched = kt.batched ? 1 : 0;
          ok = make_runs(uni, kt.vars, ik);
        }
        if (!ok) {
          set_error("internal: adjoint index map with more than %d runs", MAXRUN);
          return QGM_ERR_ARG;
        }
        d.m = mm;
        p->gbwd.push_back(d);
      }
    }
    // one record per RXY gate, in circuit order
    p->gparams.clear();
    for (size_t pi = 0; pi < m.param_factor.size(); ++pi) {
      const int fi = m.param_factor[pi];
      int li = -1;
      for (size_t l = 0; l < p->leaves.size(); ++l)
        if (rxy_member[l] == fi) li = (int)l;
      if (li < 0 || adj_off[li] < 0) {
        set_error("internal: parameter %zu has no adjoint", pi);
        return QGM_ERR_ARG;
      }
      GradParam g{};
      const int64_t tsz = (int64_t)p->leaves[li].table.size();
      g.dbase_off[0] = p->off_base + dbase_at[li] * 4;
      g.dbase_off[1] = p->off_base + (dbase_at[li] + 2 * tsz) * 4;
      g.adj_off = adj_off[li];
      g.adj_meta = adj_meta[li];
      g.n_int = p->leafdesc[li].n_int;
      g.n_out = p->leafdesc[li].n_out;
      g.n_slice = p->leafdesc[li].n_slice;
      for (int a = 0; a < MAXLEAFV; ++a) {
        g.out_qubit[a] = p->leafdesc[li].out_qubit[a];
        g.slice_bit[a] = p->leafdesc[li].slice_bit[a];
      }
      p->gparams.push_back(g);
    }
    p->off_gparams = gtake((int64_t)std::max<size_t>(p->gparams.size(), 1) * sizeof(GradParam));
    p->n_meta = next_meta;
    p->ws_bytes = goff + 256;
  }
  if (o.executor < 0 || o.executor > 3) {
    set_error("qgm_plan_order: bad executor %d", o.executor);
    return QGM_ERR_ARG;
  }
  if (o.resident_chunk != 0 && o.resident_chunk != 1 && o.resident_chunk != 2 &&
      o.resident_chunk != 4 && o.resident_chunk != 8) {
    set_error("qgm_plan_order: resident_chunk must be 0, 1, 2, 4 or 8");
    return QGM_ERR_ARG;
  }
  if (o.executor == QGM_EXEC_RESIDENT && p->resident.empty()) {
    set_error("qgm_plan_order: the resident executor needs a batch plan without slices whose "
              "per-bitstring live set fits in shared memory");
    return QGM_ERR_ARG;
  }
  return QGM_OK;
}

}  // namespace qgm

using namespace qgm;

// ===================================================================== C ABI
extern "C" {

const char *qgm_last_error(void) { return g_last_error.c_str(); }

int qgm_circuit_grid(int rows, int cols, int depth, uint64_t seed, int param_mode,
                     qgm_circuit **out) {
  if (!out || rows < 1 || cols < 1 || depth < 1 || rows * cols > 64) {
    set_error("qgm_circuit_grid: need rows, cols, depth >= 1 and rows*cols <= 64");
    return QGM_ERR_ARG;
  }
  *out = new qgm_circuit{grid_circuit(rows, cols, depth, seed, param_mode)};
  return QGM_OK;
}

int qgm_circuit_from_gates(int n_qubits, const qgm_gate *gates, int64_t n_gates,
                           qgm_circuit **out) {
  if (!out || n_qubits < 1 || n_qubits > 64 || n_gates < 0 || (n_gates > 0 && !gates)) {
    set_error("qgm_circuit_from_gates: bad arguments");
    return QGM_ERR_ARG;
  }
  Circuit c;
  c.n = n_qubits;
  for (int64_t i = 0; i < n_gates; ++i) {
    const qgm_gate &g = gates[i];
    bool ok = g.kind >= QGM_GATE_H && g.kind <= QGM_GATE_RXY && g.q0 >= 0 && g.q0 < n_qubits;
    if (g.kind == QGM_GATE_CZ) ok = ok && g.q1 >= 0 && g.q1 < n_qubits && g.q1 != g.q0;
    if (!ok) {
      set_error("qgm_circuit_from_gates: gate %lld is invalid", (long long)i);
      return QGM_ERR_ARG;
    }
    if (g.kind == QGM_GATE_RXY) c.param_gates.push_back((int)i);
    c.gates.push_back(g);
    c.depth = std::max(c.depth, g.cycle + 1);
  }
  c.param = !c.param_gates.empty();
  *out = new qgm_circuit{c};
  return QGM_OK;
}

int qgm_circuit_gates(const qgm_circuit *c, qgm_gate *gates, int64_t cap, int64_t *n) {
  if (!c || !n) {
    set_error("qgm_circuit_gates: null argument");
    return QGM_ERR_ARG;
  }
  *n = (int64_t)c->c.gates.size();
  if (gates)
    for (int64_t i = 0; i < std::min(cap, *n); ++i) gates[i] = c->c.gates[i];
  return QGM_OK;
}

int qgm_circuit_param_gates(const qgm_circuit *c, int32_t *idx, int64_t cap, int64_t *n) {
  if (!c || !n) {
    set_error("qgm_circuit_param_gates: null argument");
    return QGM_ERR_ARG;
  }
  *n = (int64_t)c->c.param_gates.size();
  if (idx)
    for (int64_t i = 0; i < std::min(cap, *n); ++i) idx[i] = c->c.param_gates[i];
  return QGM_OK;
}

// Expectation value <0|U^dagger O U|0> of a Pauli string O (Sec. III): the
// gates outside O's backward light cone meet their inverses and cancel;
// what remains, V, gives <0|V^dagger O V|0>, an amplitude (of the all-zero
// bitstring) of the circuit V, then O, then V^dagger, on the qubits V
// touches.  Every gate is written with the existing gate set, exactly:
// Z = T^4, X = i RXY(pi, 0), Y = i RXY(pi, pi/2), H^-1 = H, CZ^-1 = CZ,
// T^-1 = T^7, (X^1/2)^-1 = RXY(pi/2, pi), (Y^1/2)^-1 = RXY(pi/2, 3pi/2),
// RXY(theta, phi)^-1 = RXY(theta, phi + pi); the factors i go to *phase.
int qgm_circuit_observable(const qgm_circuit *c, const char *pauli, qgm_circuit **out, double *phase,
                           int32_t *qubit_of) {
  if (!c || !pauli || !out || !phase) {
    set_error("qgm_circuit_observable: null argument");
    return QGM_ERR_ARG;
  }
  const Circuit &C = c->c;
  if ((int)strlen(pauli) != C.n) {
    set_error("qgm_circuit_observable: need one Pauli character per qubit (%d)", C.n);
    return QGM_ERR_ARG;
  }
  std::vector<char> in_s(C.n, 0);
  bool any = false;
  for (int j = 0; j < C.n; ++j) {
    const char ch = pauli[j];
    if (ch != 'I' && ch != 'X' && ch != 'Y' && ch != 'Z') {
      set_error("qgm_circuit_observable: character %d is not one of I, X, Y, Z", j);
      return QGM_ERR_ARG;
    }
    in_s[j] = ch != 'I';
    any |= in_s[j];
  }
  phase[0] = 1.0;
  phase[1] = 0.0;
  *out = nullptr;
  if (!any) return QGM_OK;  // <I> = 1
  std::vector<char> keep(C.gates.size(), 0);
  for (int gi = (int)C.gates.size() - 1; gi >= 0; --gi) {
    const qgm_gate &g = C.gates[gi];
    const bool two = g.kind == QGM_GATE_CZ;
    if (in_s[g.q0] || (two && in_s[g.q1])) {
      keep[gi] = 1;
      in_s[g.q0] = 1;
      if (two) in_s[g.q1] = 1;
    }
  }
  std::vector<int> map(C.n, -1);
  int nq = 0;
  for (int j = 0; j < C.n; ++j)
    if (in_s[j]) map[j] = nq++;
  if (qubit_of)
    for (int j = 0; j < C.n; ++j) qubit_of[j] = map[j];
  std::vector<qgm_gate> w;
  auto push = [&](int kind, int cyc, int q0, int q1, double th, double ph) {
    qgm_gate g{};
    g.kind = kind;
    g.cycle = cyc;
    g.q0 = q0;
    g.q1 = q1;
    g.theta = th;
    g.phi = ph;
    w.push_back(g);
  };
  const int d = C.depth;
  for (size_t gi = 0; gi < C.gates.size(); ++gi) {
    if (!keep[gi]) continue;
    const qgm_gate &g = C.gates[gi];
    push(g.kind, g.cycle, map[g.q0], g.kind == QGM_GATE_CZ ? map[g.q1] : -1, g.theta, g.phi);
  }
  int n_i = 0;
  for (int j = 0; j < C.n; ++j) {
    switch (pauli[j]) {
      case 'Z':
        for (int r = 0; r < 4; ++r) push(QGM_GATE_T, d, map[j], -1, 0, 0);
        break;
      case 'X':
        push(QGM_GATE_RXY, d, map[j], -1, M_PI, 0.0);
        ++n_i;
        break;
      case 'Y':
        push(QGM_GATE_RXY, d, map[j], -1, M_PI, M_PI / 2);
        ++n_i;
        break;
      default:
        break;
    }
  }
  for (int gi = (int)C.gates.size() - 1; gi >= 0; --gi) {
    if (!keep[gi]) continue;
    const qgm_gate &g = C.gates[gi];
    const int cyc = 2 * d - g.cycle, q0 = map[g.q0];
    switch (g.kind) {
      case QGM_GATE_H: push(QGM_GATE_H, cyc, q0, -1, 0, 0); break;
      case QGM_GATE_CZ: push(QGM_GATE_CZ, cyc, q0, map[g.q1], 0, 0); break;
      case QGM_GATE_T:
        for (int r = 0; r < 7; ++r) push(QGM_GATE_T, cyc, q0, -1, 0, 0);
        break;
      case QGM_GATE_X12: push(QGM_GATE_RXY, cyc, q0, -1, M_PI / 2, M_PI); break;
      case QGM_GATE_Y12: push(QGM_GATE_RXY, cyc, q0, -1, M_PI / 2, 1.5 * M_PI); break;
      default: push(QGM_GATE_RXY, cyc, q0, -1, g.theta, g.phi + M_PI); break;
    }
  }
  // i^n_i
  static const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
  phase[0] = re[n_i & 3];
  phase[1] = im[n_i & 3];
  return qgm_circuit_from_gates(nq, w.data(), (int64_t)w.size(), out);
}

// App. E: the circuit as a tensor network, one tensor per gate.  Its wire
// segments between two gates are the vertices of the line graph, numbered in
// the order their consumers close them (gate order, first qubit first);
// segments sharing a gate are adjacent (a clique per gate).  Segments to the
// fixed input and output vectors are fixed indices and drop out, as the
// boundary variables do in the graphical model.
int qgm_circuit_line_graph_width(const qgm_circuit *c, int32_t *n_segments, int32_t *max_clique) {
  if (!c || !max_clique) {
    set_error("qgm_circuit_line_graph_width: null argument");
    return QGM_ERR_ARG;
  }
  const Circuit &C = c->c;
  std::vector<int> last(C.n, -1);
  std::vector<std::vector<int>> at_gate(C.gates.size());
  int ns = 0;
  for (size_t gi = 0; gi < C.gates.size(); ++gi) {
    const qgm_gate &g = C.gates[gi];
    for (int q : {g.q0, g.q1}) {
      if (q < 0 || q >= C.n || (q == g.q1 && g.q1 == g.q0)) continue;
      if (last[q] >= 0) {
        at_gate[last[q]].push_back(ns);
        at_gate[gi].push_back(ns);
        ++ns;
      }
      last[q] = (int)gi;
    }
  }
  Graph g(ns);
  for (int v = 0; v < ns; ++v) g.alive[v] = 1;
  for (const auto &segs : at_gate)
    for (size_t a = 0; a < segs.size(); ++a)
      for (size_t b = a + 1; b < segs.size(); ++b) g.add(segs[a], segs[b]);
  const std::vector<int> order = order_minfill(g, std::vector<char>(ns, 0));
  int w = 0;
  for (int v : order) w = std::max(w, g.eliminate(v));
  if (n_segments) *n_segments = ns;
  *max_clique = w;
  return QGM_OK;
}

void qgm_circuit_free(qgm_circuit *c) { delete c; }

int qgm_build_model(const qgm_circuit *c, qgm_model **out) {
  if (!c || !out) {
    set_error("qgm_build_model: null argument");
    return QGM_ERR_ARG;
  }
  qgm_model *m = new qgm_model;
  build_model(c->c, m->m);
  *out = m;
  return QGM_OK;
}

int qgm_model_get_info(const qgm_model *m, qgm_model_info *info) {
  if (!m || !info) {
    set_error("qgm_model_get_info: null argument");
    return QGM_ERR_ARG;
  }
  info->n_qubits = m->m.n;
  info->n_vars = m->m.n_vars;
  info->n_factors = (int32_t)m->m.factors.size();
  info->n_nondiag = m->m.L;
  info->n_params = 2 * (int32_t)m->m.param_factor.size();
  return QGM_OK;
}

int qgm_model_vars(const qgm_model *m, int32_t *qubit, int32_t *k) {
  if (!m || !qubit || !k) {
    set_error("qgm_model_vars: null argument");
    return QGM_ERR_ARG;
  }
  for (int v = 0; v < m->m.n_vars; ++v) {
    qubit[v] = m->m.var_qubit[v];
    k[v] = m->m.var_k[v];
  }
  return QGM_OK;
}

int qgm_model_factors(const qgm_model *m, int32_t *nvar, int32_t *scope) {
  if (!m || !nvar || !scope) {
    set_error("qgm_model_factors: null argument");
    return QGM_ERR_ARG;
  }
  for (size_t f = 0; f < m->m.factors.size(); ++f) {
    nvar[f] = m->m.factors[f].nv;
    scope[2 * f] = m->m.factors[f].v[0];
    scope[2 * f + 1] = m->m.factors[f].nv > 1 ? m->m.factors[f].v[1] : -1;
  }
  return QGM_OK;
}

void qgm_model_free(qgm_model *m) { delete m; }

void qgm_exec_release(qgm_plan *p);  // exec.cu

int qgm_plan_order(const qgm_model *m, const qgm_plan_opts *opts, qgm_plan **out) {
  if (!m || !opts || !out) {
    set_error("qgm_plan_order: null argument");
    return QGM_ERR_ARG;
  }
  qgm_plan *p = new qgm_plan;
  int rc = build_plan(m->m, *opts, p);
  if (rc != QGM_OK) {
    delete p;
    return rc;
  }
  // trees = 0 (automatic): a batch plan that no resident layout fits runs
  // stepwise, out of device memory, where contraction trees pay when they
  // save a clear share of the products
  if (opts->trees == 0 && opts->output_mode == QGM_OUT_BATCH && p->resident.empty() && !p->grad) {
    qgm_plan_opts o2 = *opts;
    o2.trees = 1;
    qgm_plan *t = new qgm_plan;
    // work weighted by where it runs: products of a tensor-core GEMM step
    // count 1/16 (split FP16 runs them more than an order of magnitude
    // faster than the FP32 product-sum kernels)
    auto weighted = [](const qgm_plan *q) {
      double w = 0;
      for (size_t si = 0; si < q->steps.size() && si < q->sim.steps.size(); ++si) {
        const StepDesc &d = q->steps[si];
        const bool tc = d.gemm >= 0 && q->gemm_tc && gemm_tc_eligible(q->gemms[d.gemm], q->Bp);
        w += q->sim.steps[si].flops * (tc ? 1.0 / 16.0 : 1.0);
      }
      return w;
    };
    if (build_plan(m->m, o2, t) == QGM_OK && weighted(t) < 0.9 * weighted(p) &&
        t->ws_bytes <= std::max<int64_t>(2 * p->ws_bytes, p->ws_bytes + ((int64_t)4 << 30))) {
      delete p;
      p = t;
    } else {
      delete t;
    }
  }
  *out = p;
  return QGM_OK;
}

int qgm_plan_get_info(const qgm_plan *p, qgm_plan_info *info) {
  if (!p || !info) {
    set_error("qgm_plan_get_info: null argument");
    return QGM_ERR_ARG;
  }
  info->order_kind = p->order_kind;
  info->n_free = (int32_t)p->order.size();
  info->max_clique = p->sim.max_clique;
  info->n_steps = (int32_t)p->steps.size();
  info->n_slice_vars = (int32_t)p->slice_vars.size();
  info->batch_padded = p->Bp;
  info->n_slices = (int64_t)1 << p->slice_vars.size();
  info->max_tensor_entries = p->sim.max_entries;
  info->workspace_bytes = p->ws_bytes;
  info->arena_bytes = p->sim.arena_peak;
  info->bytes_per_slice = p->sim.bytes;
  info->flops_per_slice = p->sim.flops;
  info->max_step_bytes = p->sim.max_step_bytes;
  info->n_gemm_steps = (int32_t)p->gemms.size();
  info->n_tile_steps = 0;
  for (const StepDesc &d : p->steps) info->n_tile_steps += d.tile_t > 0;
  info->n_nested_steps = 0;
  for (const StepRec &st : p->sim.steps) info->n_nested_steps += st.k_inner > 0;
  info->n_gemm_tc_steps = 0;
  if (p->gemm_tc)
    for (const GemmDesc &g : p->gemms) info->n_gemm_tc_steps += gemm_tc_eligible(g, p->Bp);
  return QGM_OK;
}

int qgm_plan_get_order(const qgm_plan *p, int32_t *order, int64_t cap, int64_t *n) {
  if (!p || !n) {
    set_error("qgm_plan_get_order: null argument");
    return QGM_ERR_ARG;
  }
  *n = (int64_t)p->order.size();
  if (order)
    for (int64_t i = 0; i < std::min(cap, *n); ++i) order[i] = p->order[i];
  return QGM_OK;
}

int qgm_plan_get_slice_vars(const qgm_plan *p, int32_t *vars, int64_t cap, int64_t *n) {
  if (!p || !n) {
    set_error("qgm_plan_get_slice_vars: null argument");
    return QGM_ERR_ARG;
  }
  *n = (int64_t)p->slice_vars.size();
  if (vars)
    for (int64_t i = 0; i < std::min(cap, *n); ++i) vars[i] = p->slice_vars[i];
  return QGM_OK;
}

int qgm_plan_get_steps(const qgm_plan *p, int32_t *out_rank, int32_t *k, int32_t *n_in,
                       int32_t *batched, int64_t cap) {
  if (!p) {
    set_error("qgm_plan_get_steps: null argument");
    return QGM_ERR_ARG;
  }
  for (int64_t s = 0; s < std::min<int64_t>(cap, (int64_t)p->steps.size()); ++s) {
    if (out_rank) out_rank[s] = p->steps[s].w_out;
    if (k) k[s] = p->steps[s].k;
    if (n_in) n_in[s] = p->steps[s].m;
    if (batched) batched[s] = p->steps[s].batched_out;
  }
  return QGM_OK;
}

int qgm_plan_get_step_kernels(const qgm_plan *p, int32_t *kind, int64_t cap) {
  if (!p || !kind) {
    set_error("qgm_plan_get_step_kernels: null argument");
    return QGM_ERR_ARG;
  }
  for (int64_t s = 0; s < std::min<int64_t>(cap, (int64_t)p->steps.size()); ++s) {
    const StepDesc &d = p->steps[s];
    kind[s] = d.gemm >= 0 ? 3 : (d.tile_t > 0 ? 2 : (d.batched_out ? 1 : 0));
  }
  // steps inside a run of small batch-free steps share one single-CTA launch
  for (size_t s = 0; s < p->plain_group.size(); ++s)
    for (int32_t j = 0; j < p->plain_group[s] && (int64_t)(s + j) < cap; ++j) kind[s + j] = 4;
  return QGM_OK;
}

int qgm_plan_get_step_inputs(const qgm_plan *p, int32_t step, int32_t *rec, int64_t cap, int64_t *n) {
  if (!p || !n || step < 0 || step >= (int32_t)p->sim.steps.size()) {
    set_error("qgm_plan_get_step_inputs: bad arguments");
    return QGM_ERR_ARG;
  }
  const StepRec &s = p->sim.steps[step];
  std::vector<int32_t> out;
  out.push_back((int32_t)s.uni.size());
  out.push_back(s.k);
  out.push_back((int32_t)s.inputs.size());
  for (int id : s.inputs) {
    const SymTensor &t = p->sim.tensors[id];
    out.push_back((int32_t)t.vars.size());
    out.push_back(t.batched ? 1 : 0);
    for (int v : t.vars)
      out.push_back((int32_t)(std::find(s.uni.begin(), s.uni.end(), v) - s.uni.begin()));
  }
  *n = (int64_t)out.size();
  if (rec)
    for (int64_t i = 0; i < std::min<int64_t>(cap, *n); ++i) rec[i] = out[i];
  return QGM_OK;
}

int qgm_plan_get_tuning(const qgm_plan *p, int32_t *rec, float *ms, int64_t cap, int64_t *n) {
  if (!p || !n) {
    set_error("qgm_plan_get_tuning: null argument");
    return QGM_ERR_ARG;
  }
  int64_t c = 0;
  for (size_t s = 0; s < p->tune.size(); ++s) {
    const StepTune &t = p->tune[s];
    if (t.ms_rule <= 0.f && !t.nt_cap && !t.T && !t.conv && !t.U && !t.ps) continue;
    if (c < cap) {
      if (rec) {
        rec[6 * c] = (int32_t)s;
        rec[6 * c + 1] = t.nt_cap;
        rec[6 * c + 2] = t.T;
        rec[6 * c + 3] = t.conv;
        rec[6 * c + 4] = t.U;
        rec[6 * c + 5] = t.ps;
      }
      if (ms) {
        ms[2 * c] = t.ms_rule;
        ms[2 * c + 1] = t.ms_best;
      }
    }
    ++c;
  }
  *n = c;
  return QGM_OK;
}

int qgm_plan_get_gemm(const qgm_plan *p, int32_t *rec, int64_t cap, int64_t *n) {
  if (!p || !n) {
    set_error("qgm_plan_get_gemm: null argument");
    return QGM_ERR_ARG;
  }
  int64_t c = 0;
  for (size_t s = 0; s < p->steps.size(); ++s) {
    const StepDesc &d = p->steps[s];
    if (d.gemm < 0) continue;
    if (rec && c < cap) {
      const GemmDesc &g = p->gemms[d.gemm];
      int32_t *r = rec + 12 * c;
      r[0] = (int32_t)s;
      r[1] = g.nm;
      r[2] = g.nn;
      r[3] = g.nk;
      r[4] = g.ns;
      r[5] = g.a_bat;
      r[6] = g.b_bat;
      r[7] = g.o_bat;
      r[8] = p->gemm_tc && gemm_tc_eligible(g, p->Bp) ? 1 : 0;
      r[9] = g.o_bout;
      r[10] = g.a_bout | g.b_bout;
      r[11] = r[8] && tc_config(g, p->Bp, p->tc_planes).fold ? 1 : 0;
    }
    ++c;
  }
  *n = c;
  return QGM_OK;
}

int qgm_plan_get_step_cost(const qgm_plan *p, double *bytes, double *flops, int64_t cap) {
  if (!p) {
    set_error("qgm_plan_get_step_cost: null argument");
    return QGM_ERR_ARG;
  }
  for (int64_t s = 0; s < std::min<int64_t>(cap, (int64_t)p->sim.steps.size()); ++s) {
    if (bytes) bytes[s] = p->sim.steps[s].bytes;
    if (flops) flops[s] = p->sim.steps[s].flops;
  }
  return QGM_OK;
}

void qgm_plan_free(qgm_plan *p) {
  if (!p) return;
  qgm_exec_release(p);
  delete p;
}

}  // extern "C"

int qgm_plan_kernel_source(const qgm_plan *p, int32_t chunk, int32_t part, int32_t min_blocks, char *buf,
                           int64_t cap, int64_t *len) {
  if (!p || !len || part < RES_WHOLE || part > RES_PRE) {
    set_error("qgm_plan_kernel_source: bad argument");
    return QGM_ERR_ARG;
  }
  const ResidentLayout *L = nullptr;
  for (const ResidentLayout &l : p->resident)
    if (l.chunk == chunk) L = &l;
  if (!L) {
    set_error("qgm_plan_kernel_source: no resident layout with %d bitstrings per CTA", chunk);
    return QGM_ERR_ARG;
  }
  const int mb = min_blocks > 0 ? min_blocks
                                : (int)std::max<int64_t>(1, std::min<int64_t>(8, (228 * 1024) / (compiled_smem(*L) + 1024)));
  const std::string src = resident_source(p, *L, part == RES_PRE ? "qgm_resident_pre" : "qgm_resident_plan", mb, part);
  *len = (int64_t)src.size();
  if (buf && cap > 0) {
    const int64_t n = std::min<int64_t>(cap - 1, (int64_t)src.size());
    std::memcpy(buf, src.data(), (size_t)n);
    buf[n] = '\0';
  }
  return QGM_OK;
}
