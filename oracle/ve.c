/*
 * Bucket (variable) elimination in FP64, plain C -- TEST INFRASTRUCTURE ONLY
 * (the oracle; only tests/, the smoke check and the benchmark's CPU legs run
 * it; it shares no code with the CUDA library).
 *
 * App. A of Boixo, Isakov, Smelyanskiy, Neven (arXiv:1712.05384), written
 * from its description: a tensor is a complex function of Boolean indexes
 * kept sorted by elimination position, the first index being the earliest
 * variable; every factor goes to the bucket of its first index; buckets are
 * processed in elimination order, each one replaced by the sum over its
 * variable of the product of its tensors (Eq. par_sum); a result of rank > 0
 * goes to the bucket of its first index, a rank-0 result multiplies into the
 * answer.
 *
 * Variables with a known value (the inputs b^0 = 0 and the outputs
 * b^d = x_j of Eq. psi_x, and any variable the caller conditions on to
 * slice the sum) enter through the factors: sum_b delta(b, c) f(b, ...) =
 * f(c, ...), so each factor holding such a variable is restricted to its
 * value before elimination starts.  The caller sums sliced results.
 *
 * The product-sum of a bucket is the definition, entry by entry:
 *     out[R] = sum_{v in {0,1}} prod_i T_i[index of (v, R) in T_i]
 * computed in parallel over R (OpenMP); each thread walks its range of R in
 * increasing order and moves every operand index by the change of the bits
 * that carried (an odometer), which is the same index arithmetic written
 * incrementally.
 *
 * Parity: pinned against the state vector and the numpy bucket elimination
 * on small grids, App. D (1/2) and normalisation (tests/test_oracle_vec.py).
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
  int rank;
  int *vars; /* sorted by elimination position, vars[0] the earliest */
  cplx *data; /* 2^rank entries, vars[0] the most significant index bit */
} tensor;

typedef struct node {
  tensor t;
  struct node *next;
} node;

static void push(node **bucket, tensor t) {
  node *n = (node *)malloc(sizeof(node));
  n->t = t;
  n->next = *bucket;
  *bucket = n;
}

/* Restrict factor f (scope vars, table over them, vars[0] most significant)
 * to the values of the fixed variables, then sort its remaining variables by
 * elimination position. */
static tensor restrict_factor(int rank, const int *vars, const double *table, const int *fixed,
                              const int *pos) {
  tensor t;
  int keep[64], nk = 0;
  for (int a = 0; a < rank; ++a)
    if (fixed[vars[a]] < 0) keep[nk++] = a;
  /* keep sorted by position (insertion sort; ranks are tiny) */
  for (int i = 1; i < nk; ++i) {
    int x = keep[i], j = i - 1;
    while (j >= 0 && pos[vars[keep[j]]] > pos[vars[x]]) {
      keep[j + 1] = keep[j];
      --j;
    }
    keep[j + 1] = x;
  }
  t.rank = nk;
  t.vars = (int *)malloc(sizeof(int) * (nk > 0 ? nk : 1));
  for (int i = 0; i < nk; ++i) t.vars[i] = vars[keep[i]];
  t.data = (cplx *)malloc(sizeof(cplx) << nk);
  for (int64_t r = 0; r < ((int64_t)1 << nk); ++r) {
    /* full index into the table: fixed values, and the bits of r */
    int64_t idx = 0;
    for (int a = 0; a < rank; ++a) {
      int bit;
      if (fixed[vars[a]] >= 0) bit = fixed[vars[a]];
      else {
        int i = 0;
        while (keep[i] != a) ++i;
        bit = (int)((r >> (nk - 1 - i)) & 1);
      }
      idx |= (int64_t)bit << (rank - 1 - a);
    }
    t.data[r] = table[2 * idx] + I * table[2 * idx + 1];
  }
  return t;
}

/* Sum over variable v of the product of the tensors in `in` (n of them). */
static tensor bucket_step(int v, node *in, int n, const int *pos) {
  /* union of the variables, sorted by position; v is the earliest */
  int uni[64], nu = 0;
  for (node *p = in; p; p = p->next)
    for (int a = 0; a < p->t.rank; ++a) {
      int u = p->t.vars[a], seen = 0;
      for (int b = 0; b < nu; ++b) seen |= uni[b] == u;
      if (!seen) uni[nu++] = u;
    }
  for (int i = 1; i < nu; ++i) {
    int x = uni[i], j = i - 1;
    while (j >= 0 && pos[uni[j]] > pos[x]) {
      uni[j + 1] = uni[j];
      --j;
    }
    uni[j + 1] = x;
  }
  /* uni[0] == v; output over uni[1..nu-1].  Union index U: uni[a] at bit
   * nu-1-a.  stride[i][bit] = the step of operand i's index for that bit. */
  tensor out;
  out.rank = nu - 1;
  out.vars = (int *)malloc(sizeof(int) * (nu > 1 ? nu - 1 : 1));
  for (int a = 1; a < nu; ++a) out.vars[a - 1] = uni[a];
  const int64_t nout = (int64_t)1 << out.rank;
  out.data = (cplx *)malloc(sizeof(cplx) * nout);
  const cplx **op = (const cplx **)malloc(sizeof(cplx *) * n);
  int64_t(*stride)[64] = malloc(sizeof(int64_t[64]) * n);
  {
    int i = 0;
    for (node *p = in; p; p = p->next, ++i) {
      op[i] = p->t.data;
      for (int b = 0; b < 64; ++b) stride[i][b] = 0;
      for (int a = 0; a < p->t.rank; ++a) {
        int ua = 0;
        while (uni[ua] != p->t.vars[a]) ++ua;
        stride[i][nu - 1 - ua] = (int64_t)1 << (p->t.rank - 1 - a);
      }
    }
  }
  const int rb = out.rank; /* bits of R: union bits 0 .. rb-1; v is bit rb */
#pragma omp parallel if (nout >= 16384)
  {
    int nt = 1, tid = 0;
#ifdef _OPENMP
    nt = omp_get_num_threads();
    tid = omp_get_thread_num();
#endif
    const int64_t r0 = nout * tid / nt, r1 = nout * (tid + 1) / nt;
    int64_t idx[64];
    for (int i = 0; i < n; ++i) {
      idx[i] = 0;
      for (int b = 0; b < rb; ++b)
        if ((r0 >> b) & 1) idx[i] += stride[i][b];
    }
    for (int64_t r = r0; r < r1; ++r) {
      if (r > r0) {
        /* r - 1 -> r: bit t set, bits below t cleared */
        const int t = __builtin_ctzll((unsigned long long)r);
        for (int i = 0; i < n; ++i) {
          int64_t d = stride[i][t];
          for (int b = 0; b < t; ++b) d -= stride[i][b];
          idx[i] += d;
        }
      }
      cplx acc = 0;
      for (int e = 0; e < 2; ++e) {
        cplx prod = 1;
        for (int i = 0; i < n; ++i) prod *= op[i][idx[i] + (e ? stride[i][rb] : 0)];
        acc += prod;
      }
      out.data[r] = acc;
    }
  }
  free(op);
  free(stride);
  return out;
}

/*
 * Amplitude of one configuration of the fixed variables.
 *  n_vars         variables of the model
 *  n_factors      gate factors; factor f has rank[f] variables
 *                 vars[off[f] .. off[f]+rank[f]-1] and a table of 2^rank
 *                 complex entries at tables[2*toff[f] ...] (re, im), the
 *                 first variable the most significant index bit
 *  fixed[v]       -1 for a variable to eliminate, else its value (0 or 1)
 *  order, n_order elimination order of the free variables
 *  threads        OpenMP threads (0 = the runtime's default)
 *  out            the complex result (re, im)
 * Returns 0, or -1 when a free variable is missing from the order.
 */
int ve_amplitude(int n_vars, int n_factors, const int *rank, const int64_t *off, const int *vars,
                 const int64_t *toff, const double *tables, const int *fixed, const int *order, int n_order,
                 int threads, double *out) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
  int *pos = (int *)malloc(sizeof(int) * n_vars);
  for (int v = 0; v < n_vars; ++v) pos[v] = -1;
  for (int i = 0; i < n_order; ++i) pos[order[i]] = i;
  for (int v = 0; v < n_vars; ++v)
    if (fixed[v] < 0 && pos[v] < 0) {
      free(pos);
      return -1;
    }
  node **bucket = (node **)calloc(n_vars, sizeof(node *));
  cplx result = 1;
  for (int f = 0; f < n_factors; ++f) {
    tensor t = restrict_factor(rank[f], vars + off[f], tables + 2 * toff[f], fixed, pos);
    if (t.rank == 0) {
      result *= t.data[0];
      free(t.vars);
      free(t.data);
    } else {
      push(&bucket[t.vars[0]], t);
    }
  }
  for (int i = 0; i < n_order; ++i) {
    const int v = order[i];
    node *in = bucket[v];
    bucket[v] = NULL;
    if (!in) {
      /* a variable no factor holds: the sum over it doubles the result */
      result *= 2;
      continue;
    }
    int n = 0;
    for (node *p = in; p; p = p->next) ++n;
    tensor t = bucket_step(v, in, n, pos);
    while (in) {
      node *nx = in->next;
      free(in->t.vars);
      free(in->t.data);
      free(in);
      in = nx;
    }
    if (t.rank == 0) {
      result *= t.data[0];
      free(t.vars);
      free(t.data);
    } else {
      push(&bucket[t.vars[0]], t);
    }
  }
  free(bucket);
  free(pos);
  out[0] = creal(result);
  out[1] = cimag(result);
  return 0;
}
