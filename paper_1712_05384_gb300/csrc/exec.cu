// Device execution of an elimination plan on sm_103a.
//
// Every tensor is a complex function of Boolean variables kept sorted by
// elimination position, the earliest variable in the most significant index
// bit (the paper's App. A invariant: indexes ordered low to high, sum over the
// first axis).  A tensor that depends on the output bitstring carries a batch
// axis beta as its innermost, contiguous dimension: row r holds the values of
// all batch entries for variable assignment r.  One elimination step of
// Eq. par_sum (a bucket of App. A, possibly several consecutive buckets fused)
// is
//
//     out[j][beta] = sum_{e in {0,1}^k} prod_i F_i[pext(e.j, mask_i)][beta]
//
// where e.j is the union index (summed variables on top) and pext drops the
// bits of variables F_i does not hold.  Because beta is innermost, every load
// of a batched operand is a coalesced 128-bit load of two complex64 values,
// whatever the variable order; gate factors without beta are tiny and hit L1.
//
// Amplitudes shrink like 2^{-n/2} and intermediate sums grow with the number
// of paths, so each intermediate tensor carries a power-of-two exponent: the
// producing kernel records max(|re|,|im|) over the tensor; the consuming
// kernel scales that operand by 2^{-e} (exact) with e = floor(log2 max) + 1
// and adds e to the exponent it passes on.  Partial amplitudes of the slices
// are summed in FP64 with their exponents applied.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "host.h"

using namespace qgm;

namespace {

struct Header {
  int32_t status;    // QGM_OK or a QGM_ERR_* code raised on the device
  int32_t slice_id;  // slice being computed
  int32_t pad[62];
};

struct Meta {
  uint32_t maxbits;  // float bits of max(|re|, |im|) over the tensor (>= 0)
  int32_t exp;       // the tensor's values are multiplied by 2^exp
};

constexpr int STEP_THREADS = 128;

// Power-of-two rescale of an operand from its recorded maximum.  For a normal
// maximum with biased exponent E, max in [2^(E-127), 2^(E-126)), so
// e = E - 126 puts the scaled maximum in [0.5, 1).
__device__ __forceinline__ void operand_scale(const Meta *meta, int slot, Header *hdr, float *scale,
                                              int *e_out) {
  if (slot < 0) {
    *scale = 1.f;
    *e_out = 0;
    return;
  }
  uint32_t bits = meta[slot].maxbits;
  int E = (int)((bits >> 23) & 0xff);
  if (E == 0xff) {
    if (hdr) atomicCAS(&hdr->status, 0, QGM_ERR_NONFINITE);
    *scale = 1.f;
    *e_out = 0;
    return;
  }
  if (E == 0) {  // zero (or a subnormal maximum): leave as is
    *scale = 1.f;
    *e_out = 0;
    return;
  }
  int e = E - 126;
  if (e > 126) e = 126;
  *scale = __int_as_float((127 - e) << 23);
  *e_out = e;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Maximum that keeps NaN (fmaxf would drop it): a NaN entry must reach the
// tensor's recorded maximum so that the consumer flags QGM_ERR_NONFINITE.
// NaN's bit pattern also orders above every finite value and Inf as unsigned.
__device__ __forceinline__ float fmax_nan(float a, float b) { return (a > b || a != a) ? a : b; }

__device__ __forceinline__ float absmax2(float2 a) { return fmax_nan(fabsf(a.x), fabsf(a.y)); }

// Block-wide max of non-negative floats, then one atomicMax on the slot
// (non-negative IEEE floats order like their unsigned bit patterns).
__device__ __forceinline__ void record_max(float v, Meta *meta, int slot) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, wid = t >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    v = lane < nw ? red[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmax_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0 && (v > 0.f || v != v)) atomicMax(&meta[slot].maxbits, __float_as_uint(v));
  }
}

// Leaf factors for the current slice and batch: base table entry chosen by
// the leaf's internal row, the slice bits and the output bits of x_beta.
// One block per leaf; block 0 also clears the intermediate metadata.
__global__ void k_build_leaves(char *ws, const LeafDesc *leaves, int n_leaves, Meta *meta,
                               int n_meta, const Header *hdr, const uint64_t *bits, int64_t B,
                               int Bp) {
  const int li = blockIdx.x;
  if (li == 0)
    for (int i = threadIdx.x; i < n_meta; i += blockDim.x) {
      meta[i].maxbits = 0;
      meta[i].exp = 0;
    }
  if (li >= n_leaves) return;
  const LeafDesc d = leaves[li];
  const int slice = hdr->slice_id;
  int sbits = 0;
  for (int a = 0; a < d.n_slice; ++a) sbits |= ((slice >> d.slice_bit[a]) & 1) << (d.n_slice - 1 - a);
  const float2 *base = reinterpret_cast<const float2 *>(ws + d.base_off);
  float2 *out = reinterpret_cast<float2 *>(ws + d.out_off);
  const int rows = 1 << d.n_int;
  const int width = d.batched ? Bp : 1;
  for (int t = threadIdx.x; t < rows * width; t += blockDim.x) {
    const int r = t / width, b = t - r * width;
    int obits = 0;
    if (d.n_out > 0) {
      const uint64_t x = (b < B) ? bits[b] : 0ull;
      for (int a = 0; a < d.n_out; ++a)
        obits |= (int)((x >> d.out_qubit[a]) & 1ull) << (d.n_out - 1 - a);
    }
    const int idx = (((r << d.n_slice) | sbits) << d.n_out) | obits;
    out[t] = base[idx];
  }
}

// Position in an input's index of union bit b (from the input's runs), as
// the value 2^pos, or 0 when the input does not hold that variable.
__device__ __forceinline__ int64_t run_bit(const InDesc &in, int b) {
  for (int q = 0; q < in.nruns; ++q) {
    const int s0 = in.src[q];
    if (b >= s0 && b < s0 + in.len[q]) return (int64_t)1 << (in.dst[q] + b - s0);
  }
  return 0;
}

// Increment tables of one launch (every input index is linear in the bits of
// the union index): when a thread's row counter carries into bit t the byte
// address of input i moves by rowtab[i][t]; when its term counter carries into
// bit t, by etab[i][t].  Rows advance by 2^r0, terms by 2^lt.
constexpr int ROWTAB = 32, ETAB = 16;

__device__ void build_tables(const StepDesc &d, int r0, int lt, int Bp, int64_t (*rowtab)[ROWTAB],
                             int64_t (*etab)[ETAB], int tid, int nthreads) {
  for (int x = tid; x < MAXIN * (ROWTAB + ETAB); x += nthreads) {
    const int i = x / (ROWTAB + ETAB), t = x - i * (ROWTAB + ETAB);
    if (i >= d.m) continue;
    const InDesc &in = d.in[i];
    const int64_t unit = in.batched ? (int64_t)Bp * 8 : 8;
    const bool row = t < ROWTAB;
    const int tt = row ? t : t - ROWTAB;
    const int base = row ? r0 : d.w_out + lt;
    const int lim = row ? d.w_out - r0 : d.k - lt;
    int64_t v = 0;
    if (tt < lim) {
      v = run_bit(in, base + tt);
      for (int b = 0; b < tt; ++b) v -= run_bit(in, base + b);
    }
    if (row) rowtab[i][tt] = v * unit;
    else etab[i][tt] = v * unit;
  }
}

// Product-sum step, batched output: thread (x, y) = (pair of batch entries,
// term group).  Rows are walked at stride gridDim.y (a power of two), terms
// at stride blockDim.y (a power of two); addresses advance by table lookups.
template <int M, int U>
__global__ void __launch_bounds__(512)
    k_step_batched(char *ws, const StepDesc d, Meta *meta, Header *hdr, int Bp, int logP) {
  __shared__ float4 part[512];
  __shared__ int64_t rowtab[MAXIN][ROWTAB];
  __shared__ int64_t etab[MAXIN][ETAB];
  const int tx = threadIdx.x, ty = threadIdx.y, T = blockDim.y;
  const int tid = ty * STEP_THREADS + tx;
  // wide batch (logP < 0): a row spans gridDim.x blocks of pairs; narrow
  // batch: a block covers 128 / 2^logP rows, 2^logP pair slots each
  const int rpb_log = logP < 0 ? 0 : 7 - logP;
  const uint64_t rstride = (uint64_t)gridDim.y << rpb_log;
  const int r0 = __ffsll((long long)rstride) - 1, lt = __ffs(T) - 1;
  build_tables(d, r0, lt, Bp, rowtab, etab, tid, STEP_THREADS * T);
  const int bp = logP < 0 ? (blockIdx.x * STEP_THREADS + tx) * 2 : (tx & ((1 << logP) - 1)) * 2;
  const bool active = bp < Bp;
  float scale[M];
  int esum = 0;
  int64_t rowb[M], eb0[M];
  const uint64_t j0 = logP < 0 ? blockIdx.y : ((uint64_t)blockIdx.y << rpb_log) + (tx >> logP);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    scale[i] = 1.f;
    rowb[i] = 0;
    eb0[i] = 0;
    {
      const InDesc &in = d.in[i];
      int e;
      operand_scale(meta, in.meta, hdr, &scale[i], &e);
      esum += e + (in.meta >= 0 ? meta[in.meta].exp : 0);
      const int64_t unit = in.batched ? (int64_t)Bp * 8 : 8;
      int64_t ri = 0, ei = 0;
      for (int b = 0; b < r0 && b < d.w_out; ++b)
        if ((j0 >> b) & 1) ri += run_bit(in, b);
      for (int b = 0; b < lt; ++b)
        if ((ty >> b) & 1) ei += run_bit(in, d.w_out + b);
      rowb[i] = in.off + ri * unit + (in.batched ? (int64_t)bp * 8 : 0);
      eb0[i] = ei * unit;
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) meta[d.out_meta].exp = esum;
  __syncthreads();
  const uint64_t rows = 1ull << d.w_out;
  const int tcount = 1 << (d.k - lt);
  float lmax = 0.f;
  float2 *out = reinterpret_cast<float2 *>(ws + d.out_off);
  uint64_t it = 0;
  // every thread of the block runs the same number of row iterations (the
  // term-group reduction below synchronises the block)
  const uint64_t jb0 = logP < 0 ? j0 : ((uint64_t)blockIdx.y << rpb_log);
  for (uint64_t jb = jb0; jb < rows; jb += rstride, ++it) {
    const uint64_t j = j0 + it * rstride;
    if (it) {
      const int t = __ffsll((long long)it) - 1;
#pragma unroll
      for (int i = 0; i < M; ++i)
        rowb[i] += rowtab[i][t];
    }
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
    const bool live = active && j < rows;
    if (live) {
      int64_t eb[M];
#pragma unroll
      for (int i = 0; i < M; ++i) eb[i] = eb0[i];
      if (tcount == 1) {
        float2 p0 = make_float2(1.f, 0.f), p1 = p0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          {
            const char *a = ws + rowb[i] + eb[i];
            if (d.in[i].batched) {
              const float4 v = __ldg(reinterpret_cast<const float4 *>(a));
              p0 = cmul(p0, make_float2(v.x * scale[i], v.y * scale[i]));
              p1 = cmul(p1, make_float2(v.z * scale[i], v.w * scale[i]));
            } else {
              const float2 v = __ldg(reinterpret_cast<const float2 *>(a));
              const float2 sv = make_float2(v.x * scale[i], v.y * scale[i]);
              p0 = cmul(p0, sv);
              p1 = cmul(p1, sv);
            }
          }
        }
        a0 = p0;
        a1 = p1;
      } else if (U >= 4 && tcount >= U) {
        // U = 4 or 8 terms per iteration (their loads in flight together):
        // terms jt .. jt + U - 1 differ in the log2(U) lowest term bits; bit
        // b moves the address by r_b, with r_0 = e_0, r_1 = e_0 + e_1,
        // r_2 = 2 e_0 + e_1 + e_2 (e_t: the carry-table steps)
        for (int jt = 0; jt < tcount; jt += U) {
          float2 p[U][2];
#pragma unroll
          for (int u = 0; u < U; ++u) p[u][0] = p[u][1] = make_float2(1.f, 0.f);
#pragma unroll
          for (int i = 0; i < M; ++i) {
            const int64_t r0 = etab[i][0], r1 = etab[i][0] + etab[i][1];
            const int64_t r2 = U == 8 ? 2 * etab[i][0] + etab[i][1] + etab[i][2] : 0;
            const char *a = ws + rowb[i] + eb[i];
            if (d.in[i].batched) {
              float4 v[U];
#pragma unroll
              for (int u = 0; u < U; ++u)
                v[u] = __ldg(reinterpret_cast<const float4 *>(a + ((u & 1) ? r0 : 0) + ((u & 2) ? r1 : 0) +
                                                              ((u & 4) ? r2 : 0)));
#pragma unroll
              for (int u = 0; u < U; ++u) {
                p[u][0] = cmul(p[u][0], make_float2(v[u].x * scale[i], v[u].y * scale[i]));
                p[u][1] = cmul(p[u][1], make_float2(v[u].z * scale[i], v[u].w * scale[i]));
              }
            } else {
              float2 v[U];
#pragma unroll
              for (int u = 0; u < U; ++u)
                v[u] = __ldg(reinterpret_cast<const float2 *>(a + ((u & 1) ? r0 : 0) + ((u & 2) ? r1 : 0) +
                                                              ((u & 4) ? r2 : 0)));
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const float2 sv = make_float2(v[u].x * scale[i], v[u].y * scale[i]);
                p[u][0] = cmul(p[u][0], sv);
                p[u][1] = cmul(p[u][1], sv);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            a0.x += p[u][0].x;
            a0.y += p[u][0].y;
            a1.x += p[u][1].x;
            a1.y += p[u][1].y;
          }
          if (jt + U < tcount) {
            const int t = __ffs(jt + U) - 1;
#pragma unroll
            for (int i = 0; i < M; ++i) {
              const int64_t r0 = etab[i][0], r1 = etab[i][0] + etab[i][1];
              const int64_t r2 = U == 8 ? 2 * etab[i][0] + etab[i][1] + etab[i][2] : 0;
              eb[i] += r0 + r1 + r2 + etab[i][t];
            }
          }
        }
      } else {
        // two terms per iteration (their loads in flight together): term jt
        // at eb, term jt + 1 one carry into bit 0 away
        for (int jt = 0; jt < tcount; jt += 2) {
          float2 p0 = make_float2(1.f, 0.f), p1 = p0, q0 = p0, q1 = p0;
#pragma unroll
          for (int i = 0; i < M; ++i) {
            {
              const char *a = ws + rowb[i] + eb[i];
              const char *b = a + etab[i][0];
              if (d.in[i].batched) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(a));
                const float4 w = __ldg(reinterpret_cast<const float4 *>(b));
                p0 = cmul(p0, make_float2(v.x * scale[i], v.y * scale[i]));
                p1 = cmul(p1, make_float2(v.z * scale[i], v.w * scale[i]));
                q0 = cmul(q0, make_float2(w.x * scale[i], w.y * scale[i]));
                q1 = cmul(q1, make_float2(w.z * scale[i], w.w * scale[i]));
              } else {
                const float2 v = __ldg(reinterpret_cast<const float2 *>(a));
                const float2 w = __ldg(reinterpret_cast<const float2 *>(b));
                const float2 sv = make_float2(v.x * scale[i], v.y * scale[i]);
                const float2 sw = make_float2(w.x * scale[i], w.y * scale[i]);
                p0 = cmul(p0, sv);
                p1 = cmul(p1, sv);
                q0 = cmul(q0, sw);
                q1 = cmul(q1, sw);
              }
            }
          }
          a0.x += p0.x + q0.x; a0.y += p0.y + q0.y;
          a1.x += p1.x + q1.x; a1.y += p1.y + q1.y;
          if (jt + 2 < tcount) {
            const int t = __ffs(jt + 2) - 1;
#pragma unroll
            for (int i = 0; i < M; ++i)
              eb[i] += etab[i][0] + etab[i][t];
          }
        }
      }
    }
    if (T > 1) {
      part[ty * STEP_THREADS + tx] = make_float4(a0.x, a0.y, a1.x, a1.y);
      __syncthreads();
      if (ty == 0) {
        for (int y = 1; y < T; ++y) {
          const float4 q = part[y * STEP_THREADS + tx];
          a0.x += q.x; a0.y += q.y; a1.x += q.z; a1.y += q.w;
        }
      }
      __syncthreads();
    }
    if (live && ty == 0) {
      reinterpret_cast<float4 *>(out)[(j * (uint64_t)Bp + bp) >> 1] = make_float4(a0.x, a0.y, a1.x, a1.y);
      lmax = fmax_nan(lmax, fmax_nan(absmax2(a0), absmax2(a1)));
    }
  }
  record_max(lmax, meta, d.out_meta);
}

// Product-sum step, batched output, with a register tile: the step's output
// bits that the largest input does not hold (tile_pos, t <= 3 of them) are
// enumerated inside a thread, so each loaded element of every input that
// lacks those bits serves all 2^t outputs.  Rows are counted over the other
// output bits ("outer" bits) and walked by table increments as in
// k_step_batched; one thread = one pair of batch entries (no term split).
template <int M>
__global__ void __launch_bounds__(STEP_THREADS)
    k_step_tile(char *ws, const StepDesc d, Meta *meta, Header *hdr, int Bp, int logP) {
  __shared__ int64_t rowtab[MAXIN][ROWTAB];
  __shared__ int64_t etab[MAXIN][ETAB];
  __shared__ int64_t toff[MAXIN][8];
  __shared__ int64_t outtab[ROWTAB];
  __shared__ int64_t tout[8];
  __shared__ int32_t tile_in[MAXIN];
  __shared__ uint8_t obits[64];
  const int tx = threadIdx.x;
  const int t = d.tile_t, ncomb = 1 << t;
  const int w_eff = d.w_out - t;
  if (tx == 0) {
    int c = 0;
    for (int b = 0; b < d.w_out; ++b) {
      bool tile = false;
      for (int q = 0; q < t; ++q) tile |= d.tile_pos[q] == b;
      if (!tile) obits[c++] = (uint8_t)b;
    }
  }
  __syncthreads();
  const int rpb_log = logP < 0 ? 0 : 7 - logP;
  const uint64_t rstride = (uint64_t)gridDim.y << rpb_log;
  const int r0 = __ffsll((long long)rstride) - 1;
  // tables over the outer bits, the summed bits, and the tile combinations
  for (int x = tx; x < MAXIN * (ROWTAB + ETAB + 8); x += STEP_THREADS) {
    const int i = x / (ROWTAB + ETAB + 8), q = x - i * (ROWTAB + ETAB + 8);
    if (i >= d.m) continue;
    const InDesc &in = d.in[i];
    const int64_t unit = in.batched ? (int64_t)Bp * 8 : 8;
    int64_t v = 0;
    if (q < ROWTAB) {
      if (q < w_eff - r0) {
        v = run_bit(in, obits[r0 + q]);
        for (int b = 0; b < q; ++b) v -= run_bit(in, obits[r0 + b]);
      }
      rowtab[i][q] = v * unit;
    } else if (q < ROWTAB + ETAB) {
      const int tt = q - ROWTAB;
      if (tt < d.k) {
        v = run_bit(in, d.w_out + tt);
        for (int b = 0; b < tt; ++b) v -= run_bit(in, d.w_out + b);
      }
      etab[i][tt] = v * unit;
    } else {
      const int c = q - ROWTAB - ETAB;
      for (int b = 0; b < t; ++b)
        if ((c >> b) & 1) v += run_bit(in, d.tile_pos[b]);
      toff[i][c] = v * unit;
    }
  }
  if (tx < ROWTAB) {
    int64_t v = 0;
    if (tx < w_eff - r0) {
      v = (int64_t)1 << obits[r0 + tx];
      for (int b = 0; b < tx; ++b) v -= (int64_t)1 << obits[r0 + b];
    }
    outtab[tx] = v * (int64_t)Bp * 8;
  } else if (tx < ROWTAB + 8) {
    const int c = tx - ROWTAB;
    int64_t v = 0;
    for (int b = 0; b < t; ++b)
      if ((c >> b) & 1) v += (int64_t)1 << d.tile_pos[b];
    tout[c] = v * (int64_t)Bp * 8;
  } else if (tx < ROWTAB + 8 + MAXIN) {
    const int i = tx - ROWTAB - 8;
    int h = 0;
    if (i < d.m)
      for (int b = 0; b < t; ++b) h |= run_bit(d.in[i], d.tile_pos[b]) != 0;
    tile_in[i] = h;
  }
  const int bp = logP < 0 ? (blockIdx.x * STEP_THREADS + tx) * 2 : (tx & ((1 << logP) - 1)) * 2;
  const bool active = bp < Bp;
  float scale[M];
  int esum = 0;
  int64_t rowb[M];
  const uint64_t j0 = logP < 0 ? blockIdx.y : ((uint64_t)blockIdx.y << rpb_log) + (tx >> logP);
  __syncthreads();
  int64_t orow = 0;
  for (int b = 0; b < r0 && b < w_eff; ++b)
    if ((j0 >> b) & 1) orow += ((int64_t)1 << obits[b]) * (int64_t)Bp * 8;
  orow += (int64_t)bp * 8;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    scale[i] = 1.f;
    rowb[i] = 0;
    if (i < d.m) {
      const InDesc &in = d.in[i];
      int e;
      operand_scale(meta, in.meta, hdr, &scale[i], &e);
      esum += e + (in.meta >= 0 ? meta[in.meta].exp : 0);
      const int64_t unit = in.batched ? (int64_t)Bp * 8 : 8;
      int64_t ri = 0;
      for (int b = 0; b < r0 && b < w_eff; ++b)
        if ((j0 >> b) & 1) ri += run_bit(in, obits[b]);
      rowb[i] = in.off + ri * unit + (in.batched ? (int64_t)bp * 8 : 0);
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && tx == 0) meta[d.out_meta].exp = esum;
  const uint64_t rows = 1ull << w_eff;
  const int tcount = 1 << d.k;
  float lmax = 0.f;
  char *outb = ws + d.out_off;
  uint64_t it = 0;
  const uint64_t jb0 = logP < 0 ? j0 : ((uint64_t)blockIdx.y << rpb_log);
  for (uint64_t jb = jb0; jb < rows; jb += rstride, ++it) {
    const uint64_t j = j0 + it * rstride;
    if (it) {
      const int tb = __ffsll((long long)it) - 1;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i < d.m) rowb[i] += rowtab[i][tb];
      orow += outtab[tb];
    }
    if (!active || j >= rows) continue;
    float4 acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t eb[M];
#pragma unroll
    for (int i = 0; i < M; ++i) eb[i] = 0;
    for (int jt = 0; jt < tcount; ++jt) {
      if (jt) {
        const int tb = __ffs(jt) - 1;
#pragma unroll
        for (int i = 0; i < M; ++i)
          if (i < d.m) eb[i] += etab[i][tb];
      }
      // product of the inputs that hold no tile bit (shared by all outputs)
      float2 s0 = make_float2(1.f, 0.f), s1 = s0;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        if (i < d.m && !tile_in[i]) {
          const char *a = ws + rowb[i] + eb[i];
          if (d.in[i].batched) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(a));
            s0 = cmul(s0, make_float2(v.x * scale[i], v.y * scale[i]));
            s1 = cmul(s1, make_float2(v.z * scale[i], v.w * scale[i]));
          } else {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(a));
            const float2 sv = make_float2(v.x * scale[i], v.y * scale[i]);
            s0 = cmul(s0, sv);
            s1 = cmul(s1, sv);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c < ncomb) {
          float2 p0 = s0, p1 = s1;
#pragma unroll
          for (int i = 0; i < M; ++i) {
            if (i < d.m && tile_in[i]) {
              const char *a = ws + rowb[i] + eb[i] + toff[i][c];
              if (d.in[i].batched) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(a));
                p0 = cmul(p0, make_float2(v.x * scale[i], v.y * scale[i]));
                p1 = cmul(p1, make_float2(v.z * scale[i], v.w * scale[i]));
              } else {
                const float2 v = __ldg(reinterpret_cast<const float2 *>(a));
                const float2 sv = make_float2(v.x * scale[i], v.y * scale[i]);
                p0 = cmul(p0, sv);
                p1 = cmul(p1, sv);
              }
            }
          }
          acc[c].x += p0.x;
          acc[c].y += p0.y;
          acc[c].z += p1.x;
          acc[c].w += p1.y;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < ncomb) {
        *reinterpret_cast<float4 *>(outb + orow + tout[c]) = acc[c];
        lmax = fmax_nan(lmax, fmax_nan(fmax_nan(fabsf(acc[c].x), fabsf(acc[c].y)),
                                       fmax_nan(fabsf(acc[c].z), fabsf(acc[c].w))));
      }
    }
  }
  record_max(lmax, meta, d.out_meta);
}

// Product-sum step without a batch axis: thread = output entry j, rows walked
// at stride gridDim.x * blockDim.x (a power of two) with table increments.
template <int M>
__global__ void __launch_bounds__(256)
    k_step_plain(char *ws, const StepDesc d, Meta *meta, Header *hdr) {
  __shared__ int64_t rowtab[MAXIN][ROWTAB];
  __shared__ int64_t etab[MAXIN][ETAB];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int r0 = __ffsll((long long)stride) - 1;
  build_tables(d, r0, 0, 1, rowtab, etab, threadIdx.x, blockDim.x);
  float scale[M];
  int esum = 0;
  int64_t rowb[M];
  const uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    scale[i] = 1.f;
    rowb[i] = 0;
    if (i < d.m) {
      const InDesc &in = d.in[i];
      int e;
      operand_scale(meta, in.meta, hdr, &scale[i], &e);
      esum += e + (in.meta >= 0 ? meta[in.meta].exp : 0);
      int64_t ri = 0;
      for (int b = 0; b < r0 && b < d.w_out; ++b)
        if ((j0 >> b) & 1) ri += run_bit(in, b);
      rowb[i] = in.off + ri * 8;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) meta[d.out_meta].exp = esum;
  __syncthreads();
  const uint64_t rows = 1ull << d.w_out;
  const int tcount = 1 << d.k;
  float lmax = 0.f;
  float2 *out = reinterpret_cast<float2 *>(ws + d.out_off);
  uint64_t it = 0;
  for (uint64_t j = j0; j < rows; j += stride, ++it) {
    if (it) {
      const int t = __ffsll((long long)it) - 1;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i < d.m) rowb[i] += rowtab[i][t];
    }
    float2 a = make_float2(0.f, 0.f);
    int64_t eb[M];
#pragma unroll
    for (int i = 0; i < M; ++i) eb[i] = 0;
    for (int jt = 0; jt < tcount; ++jt) {
      if (jt) {
        const int t = __ffs(jt) - 1;
#pragma unroll
        for (int i = 0; i < M; ++i)
          if (i < d.m) eb[i] += etab[i][t];
      }
      float2 pr = make_float2(1.f, 0.f);
#pragma unroll
      for (int i = 0; i < M; ++i) {
        if (i < d.m) {
          const float2 v = __ldg(reinterpret_cast<const float2 *>(ws + rowb[i] + eb[i]));
          pr = cmul(pr, make_float2(v.x * scale[i], v.y * scale[i]));
        }
      }
      a.x += pr.x;
      a.y += pr.y;
    }
    out[j] = a;
    lmax = fmax_nan(lmax, absmax2(a));
  }
  record_max(lmax, meta, d.out_meta);
}

// A run of small product-sum steps without a batch axis in one launch of one
// CTA: the steps run in plan order, each as in k_step_plain over a stride of
// 256 rows, separated by block barriers (which make each step's outputs and
// exponent visible to the next).  Tensors written inside the launch are read
// with ordinary loads (not the read-only path); the recorded maximum of each
// output is stored by thread 0 after a block reduction, and the metadata is
// read through volatile loads, so no stale copy is used.
__global__ void __launch_bounds__(256)
    k_step_plain_group(char *ws, const StepDesc *descs, int first, int count, Meta *meta, Header *hdr) {
  __shared__ int64_t rowtab[MAXIN][ROWTAB];
  __shared__ int64_t etab[MAXIN][ETAB];
  __shared__ float red[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  volatile Meta *vm = meta;
  for (int si = first; si < first + count; ++si) {
    const StepDesc &d = descs[si];
    build_tables(d, 8, 0, 1, rowtab, etab, tid, 256);
    float scale[MAXIN];
    int esum = 0;
    int64_t rowb[MAXIN];
#pragma unroll
    for (int i = 0; i < MAXIN; ++i) {
      scale[i] = 1.f;
      rowb[i] = 0;
      if (i < d.m) {
        const InDesc &in = d.in[i];
        int e = 0;
        if (in.meta >= 0) {
          const uint32_t bits = vm[in.meta].maxbits;
          const int E = (int)((bits >> 23) & 0xff);
          if (E == 0xff) {
            if (hdr && tid == 0) atomicCAS(&hdr->status, 0, QGM_ERR_NONFINITE);
          } else if (E != 0) {
            e = E - 126 > 126 ? 126 : E - 126;
            scale[i] = __int_as_float((127 - e) << 23);
          }
          esum += e + vm[in.meta].exp;
        }
        int64_t ri = 0;
        for (int b = 0; b < 8 && b < d.w_out; ++b)
          if ((tid >> b) & 1) ri += run_bit(in, b);
        rowb[i] = in.off + ri * 8;
      }
    }
    if (tid == 0) vm[d.out_meta].exp = esum;
    __syncthreads();
    const uint64_t rows = 1ull << d.w_out;
    const int tcount = 1 << d.k;
    float lmax = 0.f;
    float2 *out = reinterpret_cast<float2 *>(ws + d.out_off);
    uint64_t it = 0;
    for (uint64_t j = tid; j < rows; j += 256, ++it) {
      if (it) {
        const int t = __ffsll((long long)it) - 1;
#pragma unroll
        for (int i = 0; i < MAXIN; ++i)
          if (i < d.m) rowb[i] += rowtab[i][t];
      }
      float2 a = make_float2(0.f, 0.f);
      int64_t eb[MAXIN];
#pragma unroll
      for (int i = 0; i < MAXIN; ++i) eb[i] = 0;
      for (int jt = 0; jt < tcount; ++jt) {
        if (jt) {
          const int t = __ffs(jt) - 1;
#pragma unroll
          for (int i = 0; i < MAXIN; ++i)
            if (i < d.m) eb[i] += etab[i][t];
        }
        float2 pr = make_float2(1.f, 0.f);
#pragma unroll
        for (int i = 0; i < MAXIN; ++i) {
          if (i < d.m) {
            const float2 v = *reinterpret_cast<const float2 *>(ws + rowb[i] + eb[i]);
            pr = cmul(pr, make_float2(v.x * scale[i], v.y * scale[i]));
          }
        }
        a.x += pr.x;
        a.y += pr.y;
      }
      out[j] = a;
      lmax = fmax_nan(lmax, absmax2(a));
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmax_nan(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if (lane == 0) red[wid] = lmax;
    __syncthreads();
    if (tid == 0) {
      float v = red[0];
      for (int w = 1; w < 8; ++w) v = fmax_nan(v, red[w]);
      if (v > 0.f || v != v) vm[d.out_meta].maxbits = __float_as_uint(v);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// GEMM-shaped step: out[s, m, n] = sum_k A[s, m, k] B[s, n, k] for each
// shared kept index s and batch entry (grid z and y), 64 x 64 output tiles
// (grid x), K in chunks of 16 staged in shared memory, a 4 x 4 complex tile
// per thread in registers.  Operand and output addresses come from the bit
// positions of the m, n, k, s variables in each tensor's own index.
constexpr int GT = 64;

__device__ __forceinline__ int64_t lin_bits(uint64_t x, const uint8_t *pos, int nb) {
  int64_t r = 0;
  for (int b = 0; b < nb; ++b)
    if ((x >> b) & 1) r += (int64_t)1 << pos[b];
  return r;
}

// GK: summed entries per shared-memory chunk (16, or 32 when K allows: half
// the barriers per product); NT: tile columns (64, or 32 when B has five
// private kept variables), NT / 16 per thread
template <int GK, int NT>
__global__ void __launch_bounds__(256) k_gemm(char *ws, const GemmDesc g, Meta *meta, Header *hdr, int Bp) {
  constexpr int TC = NT / 16;
  __shared__ float2 As[GK][GT];
  __shared__ float2 Bs[GK][NT];
  __shared__ int64_t oAm[GT], oBn[NT], oOm[GT], oOn[NT], oAk[GK], oBk[GK];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lnt = g.nn - (NT == 64 ? 6 : 5);
  const uint64_t tm = (uint64_t)blockIdx.x >> lnt, tn = (uint64_t)blockIdx.x & ((1ull << lnt) - 1);
  const int beta = blockIdx.y;
  const uint64_t sidx = blockIdx.z;
  const int64_t uA = g.a_bat ? (int64_t)Bp * 8 : 8, uB = g.b_bat ? (int64_t)Bp * 8 : 8,
                uO = g.o_bat ? (int64_t)Bp * 8 : 8;
  const int64_t baseA = g.a_off + lin_bits(sidx, g.sA, g.ns) * uA + (g.a_bat ? beta * 8 : 0);
  const int64_t baseB = g.b_off + lin_bits(sidx, g.sB, g.ns) * uB + (g.b_bat ? beta * 8 : 0);
  const int64_t baseO = g.o_off + lin_bits(sidx, g.sO, g.ns) * uO + (g.o_bat ? beta * 8 : 0);
  if (tid < GT) {
    oAm[tid] = lin_bits(tm * GT + tid, g.mA, g.nm) * uA;
    oOm[tid] = lin_bits(tm * GT + tid, g.mO, g.nm) * uO;
  } else if (tid < GT + NT) {
    const int j = tid - GT;
    oBn[j] = lin_bits(tn * NT + j, g.nB, g.nn) * uB;
    oOn[j] = lin_bits(tn * NT + j, g.nO, g.nn) * uO;
  }
  float sa, sb;
  int ea, eb;
  operand_scale(meta, g.a_meta, hdr, &sa, &ea);
  operand_scale(meta, g.b_meta, hdr, &sb, &eb);
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tid == 0)
    meta[g.o_meta].exp = ea + eb + (g.a_meta >= 0 ? meta[g.a_meta].exp : 0) +
                         (g.b_meta >= 0 ? meta[g.b_meta].exp : 0);
  float2 acc[4][TC];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < TC; ++c) acc[r][c] = make_float2(0.f, 0.f);
  const int nkc = (1 << g.nk) / GK;
  for (int kc = 0; kc < nkc; ++kc) {
    __syncthreads();  // the previous chunk's tiles and tables are consumed
    if (tid < GK) oAk[tid] = lin_bits((uint64_t)kc * GK + tid, g.kA, g.nk) * uA;
    else if (tid < 2 * GK) oBk[tid - GK] = lin_bits((uint64_t)kc * GK + tid - GK, g.kB, g.nk) * uB;
    __syncthreads();
    if constexpr (NT == GT) {
      // both tiles in one loop: two loads in flight per iteration
#pragma unroll
      for (int q = 0; q < GK * GT / 256; ++q) {
        const int e = tid + 256 * q, i = e & (GT - 1), j = e >> 6;
        const float2 va = __ldg(reinterpret_cast<const float2 *>(ws + baseA + oAm[i] + oAk[j]));
        const float2 vb = __ldg(reinterpret_cast<const float2 *>(ws + baseB + oBn[i] + oBk[j]));
        As[j][i] = make_float2(va.x * sa, va.y * sa);
        Bs[j][i] = make_float2(vb.x * sb, vb.y * sb);
      }
    } else {
#pragma unroll
      for (int q = 0; q < GK * GT / 256; ++q) {
        const int e = tid + 256 * q, i = e & (GT - 1), j = e >> 6;
        const float2 va = __ldg(reinterpret_cast<const float2 *>(ws + baseA + oAm[i] + oAk[j]));
        As[j][i] = make_float2(va.x * sa, va.y * sa);
      }
#pragma unroll
      for (int q = 0; q < GK * NT / 256; ++q) {
        const int e = tid + 256 * q, i = e & (NT - 1), j = e / NT;
        const float2 vb = __ldg(reinterpret_cast<const float2 *>(ws + baseB + oBn[i] + oBk[j]));
        Bs[j][i] = make_float2(vb.x * sb, vb.y * sb);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float2 a[4], b[TC];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < TC; ++c) b[c] = Bs[kk][tx * TC + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < TC; ++c) {
          acc[r][c].x = fmaf(a[r].x, b[c].x, fmaf(-a[r].y, b[c].y, acc[r][c].x));
          acc[r][c].y = fmaf(a[r].x, b[c].y, fmaf(a[r].y, b[c].x, acc[r][c].y));
        }
    }
  }
  float lmax = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < TC; ++c) {
      *reinterpret_cast<float2 *>(ws + baseO + oOm[ty * 4 + r] + oOn[tx * TC + c]) = acc[r][c];
      lmax = fmax_nan(lmax, absmax2(acc[r][c]));
    }
  record_max(lmax, meta, g.o_meta);
}

// ---------------------------------------------------------------------------
// GEMM-shaped step on the tensor cores (tcgen05.mma kind::f16, FP32
// accumulation in tensor memory) as split products of 16-bit terms.
//
// Split.  Each operand value x, scaled by a power of two from the operand's
// recorded maximum, is written as a sum of 16-bit terms once, by k_split,
// into "planes" laid out exactly as the MMA reads them (see TcCfg):
//  - FP16 (4 planes: re high, re low, im high, im low): the operand's
//    maximum is put in [2^14, 2^15) (FP16's largest value is 65504),
//    h = fp16(x) and l = fp16(x - h) (the difference is exact in FP32), so
//    x - h - l is below 2^-22 |x| (below 2^-39 of the maximum where l is
//    subnormal); a real product keeps h h' + h l' + l h', the dropped l l'
//    being below 2^-22 |x x'|: three MMAs;
//  - BF16 (6 planes: three terms of re, three of im): maximum in [0.5, 1),
//    x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) hold x exactly;
//    the six term products x_i y_j with i + j <= 2 are kept (each dropped one
//    is at most about 2^-24 |x y|): six MMAs.
// A complex product takes four real ones -- re += Ar Br - Ai Bi (the minus
// from the instruction's negate-A bit), im += Ar Bi + Ai Br -- so a chunk of
// 16 summed entries is 12 (FP16) or 24 (BF16) MMAs of 128 x NT x 16.
//
// Product.  One CTA of 128 threads per 128 x NT output tile of one instance.
// Warp 0 (one lane) streams the tile's plane blocks, one chunk per stage, with
// bulk asynchronous copies (cp.async.bulk, the TMA unit) into a ring of
// shared-memory stages, each completing a "full" mbarrier by its byte count;
// warp 1 (one lane) waits for a stage, issues its MMAs and commits them to the
// stage's "empty" mbarrier, which frees the stage for the next copy; after the
// last chunk it commits to "done".  D_re sits in tensor-memory columns
// [0, NT), D_im in [NT, 2 NT), tile row r in lane r; the four warps then read
// their 32 lanes back (tcgen05.ld), undo the terms' scale, store through the
// output's bit maps and record the maximum for the rescale.
//
// Every wait is bounded (about one second of %globaltimer).  A wait runs out
// only if a copy or an MMA never completes; the kernel then stops issuing,
// records QGM_ERR_TIMEOUT, and still ends with the MMA thread's final commit
// (tcgen05.commit tracks every MMA that thread issued), which the epilogue
// waits for before the tensor memory is released.

// Shared-memory matrix descriptor, K-major without swizzle: start address,
// leading byte offset (the next 8 summed entries: 128 B), stride byte offset
// (the next 8-row group: 256 B), descriptor version 1.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait (about one second at most) for the completion of the mbarrier phase
// of the given parity; false when the limit ran out.
__device__ __forceinline__ bool tc_wait_ns(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = gtimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) { return tc_wait_ns(bar, parity, 1000000000ull); }

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 lanes, waited for
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// Two values -> their three BF16 terms, each as a pair (first value in the
// low half: the lower address)
__device__ __forceinline__ void split3(float a, float b, uint32_t &t0, uint32_t &t1, uint32_t &t2) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const float ra = a - hf.x, rb = b - hf.y;
  const __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
  const float2 mf = __bfloat1622float2(m);
  const __nv_bfloat162 l = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
  t0 = *reinterpret_cast<const uint32_t *>(&h);
  t1 = *reinterpret_cast<const uint32_t *>(&m);
  t2 = *reinterpret_cast<const uint32_t *>(&l);
}

// Two values -> their FP16 high and low terms, each as a pair
__device__ __forceinline__ void split2h(float a, float b, uint32_t &t0, uint32_t &t1) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  t0 = *reinterpret_cast<const uint32_t *>(&h);
  t1 = *reinterpret_cast<const uint32_t *>(&l);
}

// One operand of a tensor-core step: its rows (m or n variables, batch
// entries folded in when `fold`), summed and shared variables by bit
// position in the operand's own index.
struct SplitArgs {
  int64_t src_off, dst_off;  // complex64 operand; its plane region
  int32_t meta, batched, fold, perbeta, Bp;
  int32_t nr, nk, ns;        // row, summed and shared variables
  int32_t tr;                // rows per tile (128 for the M side, NT for N)
  int64_t rows, rtiles, kc;  // rows per instance, row tiles, chunks of 16
  int32_t fp16;              // 1: FP16 terms (4 planes), 0: BF16 (6 planes)
  int32_t bout, rank;        // batch entry outermost: entry beta at beta * 2^rank complex64
  uint8_t rX[GMAXB], kX[GMAXB], sX[GMAXB];
};

// Thread = (batch entry b when per entry, row, 8 consecutive summed entries,
// shared index), b fastest, then the row: reads of neighbouring threads share
// sectors and each thread writes one 16-byte core-matrix row per plane.
template <int P>
__global__ void __launch_bounds__(256) k_split(char *ws, const __grid_constant__ SplitArgs a, Meta *meta,
                                                Header *hdr) {
  float sc;
  int e;
  operand_scale(meta, a.meta, hdr, &sc, &e);
  if (P == 4) sc *= 32768.f;  // maximum in [2^14, 2^15): FP16 terms keep 22 bits down to 2^-18 of it
  const int64_t nb = a.perbeta ? a.Bp : 1;
  const int64_t RP = a.rtiles * a.tr, KG = a.kc * 2;
  const int64_t n_items = ((int64_t)1 << a.ns) * KG * RP * nb;
  const int64_t u = a.batched && !a.bout ? (int64_t)a.Bp * 8 : 8;
  const int64_t ustride = a.bout ? ((int64_t)8 << a.rank) : 8;  // bytes between batch entries
  const int64_t pbytes = (int64_t)a.tr * 32;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n_items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = it % nb;
    int64_t t = it / nb;
    const int64_t rho = t % RP;
    t /= RP;
    const int64_t kg = t % KG;
    const int64_t s = t / KG;
    float2 v[8];
    const int klow = a.nk < 3 ? a.nk : 3;  // summed variables inside a group of 8
    if (rho < a.rows && kg * 8 < ((int64_t)1 << a.nk)) {
      const int64_t m = a.fold ? rho / a.Bp : rho;
      const int64_t beta = a.fold ? rho % a.Bp : b;
      const int64_t base = a.src_off + (lin_bits((uint64_t)s, a.sX, a.ns) + lin_bits((uint64_t)m, a.rX, a.nr) +
                                        lin_bits((uint64_t)(kg * 8), a.kX, a.nk)) * u +
                           (a.batched ? beta * ustride : 0);
      if (klow == 3) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float2 x = __ldg(reinterpret_cast<const float2 *>(ws + base + lin_bits((uint64_t)q, a.kX, 3) * u));
          v[q] = make_float2(x.x * sc, x.y * sc);
        }
      } else {
        // fewer than 8 summed entries: the rest of the group is zero padding
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q < (1 << klow)) {
            const float2 x = __ldg(reinterpret_cast<const float2 *>(ws + base + lin_bits((uint64_t)q, a.kX, klow) * u));
            v[q] = make_float2(x.x * sc, x.y * sc);
          } else {
            v[q] = make_float2(0.f, 0.f);
          }
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = make_float2(0.f, 0.f);
    }
    const int64_t inst = s * nb + b, tile = rho / a.tr, r = rho % a.tr;
    char *blk = ws + a.dst_off + ((inst * a.rtiles + tile) * a.kc + kg / 2) * (P * pbytes) + (r >> 3) * 256 +
                (kg & 1) * 128 + (r & 7) * 16;
    if (P == 4) {
      uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split2h(v[2 * q].x, v[2 * q + 1].x, rh[q], rl[q]);
        split2h(v[2 * q].y, v[2 * q + 1].y, ih[q], il[q]);
      }
      *reinterpret_cast<uint4 *>(blk) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
      *reinterpret_cast<uint4 *>(blk + pbytes) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
      *reinterpret_cast<uint4 *>(blk + 2 * pbytes) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
      *reinterpret_cast<uint4 *>(blk + 3 * pbytes) = make_uint4(il[0], il[1], il[2], il[3]);
    } else {
      uint32_t re[3][4], im[3][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split3(v[2 * q].x, v[2 * q + 1].x, re[0][q], re[1][q], re[2][q]);
        split3(v[2 * q].y, v[2 * q + 1].y, im[0][q], im[1][q], im[2][q]);
      }
#pragma unroll
      for (int t3 = 0; t3 < 3; ++t3) {
        *reinterpret_cast<uint4 *>(blk + t3 * pbytes) = make_uint4(re[t3][0], re[t3][1], re[t3][2], re[t3][3]);
        *reinterpret_cast<uint4 *>(blk + (3 + t3) * pbytes) =
            make_uint4(im[t3][0], im[t3][1], im[t3][2], im[t3][3]);
      }
    }
  }
}

// The product of a tensor-core step (after k_split of both operands).
struct TcArgs {
  int64_t pm_off, pn_off, o_off;  // plane regions of the M and N sides; output
  int32_t a_meta, b_meta, o_meta; // M side, N side, output
  int32_t o_bat, fold, perbeta, Bp;
  int32_t o_bout, o_rank;         // output batch entry outermost (2^o_rank complex64 per entry)
  int32_t s_fast;                 // shared index fastest in the grid (its bits share output sectors)
  int32_t nM, nN, ns;
  int64_t mrows, mtiles, ntiles, kc;
  float out_scale;                // undoes the terms' scale: 2^-30 (FP16) or 1
  uint8_t mO[GMAXB], nO[GMAXB], sO[GMAXB];
  // k_gemm_tc_conv: the M side read as complex64 from the operand itself
  int64_t a_src_off;
  int32_t a_batched, a_bout, a_rank, nk;
  uint8_t mA[GMAXB], kA[GMAXB], sA[GMAXB];
};

__host__ __device__ constexpr int tc_plane_bytes(int rows) { return rows * 32; }
// stages of the copy ring: up to four, within 220 KB (one CTA per SM) for
// 256-column tiles and 110 KB (two CTAs per SM) for narrower ones
__host__ __device__ constexpr int tc_stages(int nt, int planes) {
  return (nt == 256 ? 220 : 110) * 1024 / (planes * tc_plane_bytes(TC_M + nt)) < 4
             ? (nt == 256 ? 220 : 110) * 1024 / (planes * tc_plane_bytes(TC_M + nt))
             : 4;
}
__host__ __device__ constexpr int tc_smem_bytes(int nt, int planes) {
  return tc_stages(nt, planes) * planes * (tc_plane_bytes(TC_M) + tc_plane_bytes(nt));
}
// k_gemm_tc_conv: two plane stages (the converters write one while the MMAs
// read the other), and as many stages of the raw ring (the M side's
// complex64 rows of one chunk, 128 bytes per row) as fit in 220 KB, up to 8:
// the copies run that many chunks ahead of the conversion, several
// microseconds of MMA time, which covers the DRAM latency under load
__host__ __device__ constexpr int tcc_stages(int nt, int planes) { return 2; }
__host__ __device__ constexpr int tcc_raw_stages(int nt, int planes) {
  return (220 * 1024 - tcc_stages(nt, planes) * planes * (tc_plane_bytes(TC_M) + tc_plane_bytes(nt))) /
                     (TC_M * 128) < 8
             ? (220 * 1024 - tcc_stages(nt, planes) * planes * (tc_plane_bytes(TC_M) + tc_plane_bytes(nt))) /
                   (TC_M * 128)
             : 8;
}
__host__ __device__ constexpr int tcc_smem_bytes(int nt, int planes) {
  return tcc_stages(nt, planes) * planes * (tc_plane_bytes(TC_M) + tc_plane_bytes(nt)) +
         tcc_raw_stages(nt, planes) * TC_M * 128;
}
static_assert(tcc_smem_bytes(256, 4) <= 220 * 1024 && tcc_smem_bytes(256, 6) <= 220 * 1024, "conv ring");

template <int NT, int P>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(char *ws, const __grid_constant__ TcArgs a, Meta *meta,
                                                    Header *hdr) {
  constexpr int S = tc_stages(NT, P);
  constexpr int ABYTES = P * tc_plane_bytes(TC_M), BBYTES = P * tc_plane_bytes(NT);
  constexpr int SBYTES = ABYTES + BBYTES;
  constexpr uint32_t COLS = 2 * NT < 32 ? 32 : 2 * NT;
  static_assert(S >= 2, "at least two stages");
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S], bar_done;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  __shared__ int64_t colO[NT];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile coordinates: the batch entry fastest (per-entry products of one
  // tile write the same output sectors, which then merge in L2), then the N
  // tile, the M tile and the shared index
  int64_t bid = blockIdx.x;
  int64_t beta = 0, sidx = 0;
  if (a.s_fast) {
    // the output's lowest index bits include a shared variable: the tiles of
    // neighbouring instances fill the same sectors, so they run together
    sidx = bid & ((1ll << a.ns) - 1);
    bid >>= a.ns;
  }
  if (a.perbeta) {
    beta = bid % a.Bp;
    bid /= a.Bp;
  }
  const int64_t tn = bid % a.ntiles;
  bid /= a.ntiles;
  const int64_t tm = bid % a.mtiles;
  if (!a.s_fast) sidx = bid / a.mtiles;
  const int64_t inst = a.perbeta ? sidx * a.Bp + beta : sidx;
  const int64_t uO = a.o_bat && !a.o_bout ? (int64_t)a.Bp * 8 : 8;
  const int64_t bstrideO = a.o_bout ? ((int64_t)8 << a.o_rank) : 8;  // bytes between batch entries
  for (int j = tid; j < NT; j += 128) colO[j] = lin_bits((uint64_t)(tn * NT + j), a.nO, a.nN) * uO;
  if (tid == 0) abort_flag = 0;
  float sa, sb;
  int ea, eb;
  operand_scale(meta, a.a_meta, hdr, &sa, &ea);
  operand_scale(meta, a.b_meta, hdr, &sb, &eb);
  if (blockIdx.x == 0 && tid == 0)
    meta[a.o_meta].exp = ea + eb + (a.a_meta >= 0 ? meta[a.a_meta].exp : 0) + (a.b_meta >= 0 ? meta[a.b_meta].exp : 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tbase;
  const uint32_t s0 = smem_u32(tsm);
  const int64_t kc = a.kc;
  if (warp == 0) {
    if (lane == 0) {
      // producer: one chunk (both operands' plane blocks) per stage
      const char *srcA = ws + a.pm_off + (inst * a.mtiles + tm) * kc * ABYTES;
      const char *srcB = ws + a.pn_off + (inst * a.ntiles + tn) * kc * BBYTES;
      for (int64_t k = 0; k < kc; ++k) {
        const int st = (int)(k % S);
        if (k >= S && !tc_wait(smem_u32(&bar_empty[st]), (uint32_t)((k / S) - 1) & 1u)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag) break;
        const uint32_t fb = smem_u32(&bar_full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(SBYTES) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                s0 + st * SBYTES),
            "l"(srcA + k * ABYTES), "r"(ABYTES), "r"(fb)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                s0 + st * SBYTES + ABYTES),
            "l"(srcB + k * BBYTES), "r"(BBYTES), "r"(fb)
            : "memory");
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issue.  Instruction descriptor: FP32 accumulator, FP16 (P = 4)
      // or BF16 (P = 6) A and B, both K-major, N >> 3 at bit 17, M >> 4 at
      // bit 24; bit 13 negates A.
      constexpr uint32_t fmt = P == 4 ? 0u : 1u;
      constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                 ((uint32_t)(TC_M >> 4) << 24);
      constexpr uint32_t idesc_neg = idesc | (1u << 13);
      for (int64_t k = 0; k < kc; ++k) {
        const int st = (int)(k % S);
        if (!tc_wait(smem_u32(&bar_full[st]), (uint32_t)(k / S) & 1u)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sA = s0 + st * SBYTES, sB = sA + ABYTES;
        uint32_t acc = k > 0 ? 1u : 0u;
        if (P == 4) {
          // planes: 0 re high, 1 re low, 2 im high, 3 im low; term pairs
          // (h, h), (h, l), (l, h)
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int i = t == 2 ? 1 : 0, j = t == 1 ? 1 : 0;
            const uint64_t ar = tc_desc(sA + i * tc_plane_bytes(TC_M)), ai = tc_desc(sA + (2 + i) * tc_plane_bytes(TC_M));
            const uint64_t br = tc_desc(sB + j * tc_plane_bytes(NT)), bi = tc_desc(sB + (2 + j) * tc_plane_bytes(NT));
            tc_mma(tmem, ar, br, idesc, acc);           // re += Ar Br
            tc_mma(tmem, ai, bi, idesc_neg, 1u);        // re -= Ai Bi
            tc_mma(tmem + NT, ar, bi, idesc, acc);      // im += Ar Bi
            tc_mma(tmem + NT, ai, br, idesc, 1u);       // im += Ai Br
            acc = 1u;
          }
        } else {
          // planes: 0-2 re terms, 3-5 im terms; term pairs (i, j), i + j <= 2
#pragma unroll
          for (int t = 0; t < 6; ++t) {
            const int i = t == 2 || t == 4 ? 1 : t == 5 ? 2 : 0;
            const int j = t == 1 || t == 4 ? 1 : t == 3 ? 2 : 0;
            const uint64_t ar = tc_desc(sA + i * tc_plane_bytes(TC_M)), ai = tc_desc(sA + (3 + i) * tc_plane_bytes(TC_M));
            const uint64_t br = tc_desc(sB + j * tc_plane_bytes(NT)), bi = tc_desc(sB + (3 + j) * tc_plane_bytes(NT));
            tc_mma(tmem, ar, br, idesc, acc);
            tc_mma(tmem, ai, bi, idesc_neg, 1u);
            tc_mma(tmem + NT, ar, bi, idesc, acc);
            tc_mma(tmem + NT, ai, br, idesc, 1u);
            acc = 1u;
          }
        }
        tc_commit(smem_u32(&bar_empty[st]));
      }
      // always: every MMA issued above completes before "done" does
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  }
  // epilogue: thread r = tile row r = tensor-memory lane r
  bool ok = tc_wait(smem_u32(&bar_done), 0u);
  if (!ok) ok = tc_wait(smem_u32(&bar_done), 0u);  // MMAs read only loaded stages: they finish
  ok = __all_sync(0xffffffffu, ok);                 // tcgen05.ld below is warp-collective
  const bool valid_run = ok && !*(volatile int *)&abort_flag;
  float lmax = 0.f;
  if (ok) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int64_t rho = tm * TC_M + tid;
    const bool valid = valid_run && rho < a.mrows;
    int64_t m = rho, b2 = beta;
    if (a.fold) {
      m = rho / a.Bp;
      b2 = rho % a.Bp;
    }
    char *orow = ws + a.o_off + (lin_bits((uint64_t)sidx, a.sO, a.ns) + lin_bits((uint64_t)(valid ? m : 0), a.mO, a.nM)) * uO +
                 (a.o_bat ? b2 * bstrideO : 0);
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t re[16], im[16];
      tc_ld16(tl + c0, re);
      tc_ld16(tl + NT + c0, im);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 v = make_float2(__uint_as_float(re[j]) * a.out_scale, __uint_as_float(im[j]) * a.out_scale);
          *reinterpret_cast<float2 *>(orow + colO[c0 + j]) = v;
          lmax = fmax_nan(lmax, absmax2(v));
        }
      }
    }
  }
  if (!valid_run && tid == 0 && hdr) atomicCAS(&hdr->status, 0, QGM_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
  record_max(lmax, meta, a.o_meta);
}

// The folded tensor-core step with the M side converted in the kernel.  When
// the batch entries fold into the M side (one operand without a batch axis),
// that side is the large operand streamed once; splitting it in a separate
// pass would read and write it once more.  Here 8 warps: warp 0 streams the
// N side's planes (bulk copies, as k_gemm_tc), warp 1 issues the MMAs, warps
// 4-7 convert: thread r copies row r of each chunk (16 complex64 values
// through the operand's bit maps) into a raw ring in shared memory with
// cp.async, RS - 1 chunks ahead, then scales and splits it into the 16-bit
// planes of the stage (the layout k_split writes), makes the stores visible
// to the tensor cores (fence.proxy.async) and arrives on the stage's "full"
// mbarrier, which completes when the 128 converters and the N side's bytes
// are in.  Warps 4-7 then read the accumulators back (TMEM lane quadrant =
// warp % 4).  Waits are bounded as in k_gemm_tc.
template <int P>
__device__ __forceinline__ void conv_put(uint8_t *stage, int r, const float2 (&v)[16]) {
  const int pb = tc_plane_bytes(TC_M);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint8_t *base = stage + (r >> 3) * 256 + half * 128 + (r & 7) * 16;
    if (P == 4) {
      uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split2h(v[half * 8 + 2 * q].x, v[half * 8 + 2 * q + 1].x, rh[q], rl[q]);
        split2h(v[half * 8 + 2 * q].y, v[half * 8 + 2 * q + 1].y, ih[q], il[q]);
      }
      *reinterpret_cast<uint4 *>(base) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
      *reinterpret_cast<uint4 *>(base + pb) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
      *reinterpret_cast<uint4 *>(base + 2 * pb) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
      *reinterpret_cast<uint4 *>(base + 3 * pb) = make_uint4(il[0], il[1], il[2], il[3]);
    } else {
      uint32_t re[3][4], im[3][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split3(v[half * 8 + 2 * q].x, v[half * 8 + 2 * q + 1].x, re[0][q], re[1][q], re[2][q]);
        split3(v[half * 8 + 2 * q].y, v[half * 8 + 2 * q + 1].y, im[0][q], im[1][q], im[2][q]);
      }
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        *reinterpret_cast<uint4 *>(base + t * pb) = make_uint4(re[t][0], re[t][1], re[t][2], re[t][3]);
        *reinterpret_cast<uint4 *>(base + (3 + t) * pb) = make_uint4(im[t][0], im[t][1], im[t][2], im[t][3]);
      }
    }
  }
}

template <int NT, int P>
__global__ void __launch_bounds__(256, 1) k_gemm_tc_conv(char *ws, const __grid_constant__ TcArgs a, Meta *meta,
                                                         Header *hdr) {
  constexpr int S = tcc_stages(NT, P), RS = tcc_raw_stages(NT, P);
  static_assert(RS >= 3, "raw ring");
  constexpr int ABYTES = P * tc_plane_bytes(TC_M), BBYTES = P * tc_plane_bytes(NT);
  constexpr int SBYTES = ABYTES + BBYTES;
  constexpr uint32_t COLS = 2 * NT < 32 ? 32 : 2 * NT;
  static_assert(S >= 2, "at least two stages");
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S], bar_done;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  __shared__ int64_t colO[NT];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int64_t bid = blockIdx.x;
  int64_t sidx = 0;
  if (a.s_fast) {
    sidx = bid & ((1ll << a.ns) - 1);
    bid >>= a.ns;
  }
  const int64_t tn = bid % a.ntiles;
  bid /= a.ntiles;
  const int64_t tm = bid % a.mtiles;
  if (!a.s_fast) sidx = bid / a.mtiles;
  const int64_t uO = a.o_bat && !a.o_bout ? (int64_t)a.Bp * 8 : 8;
  const int64_t bstrideO = a.o_bout ? ((int64_t)8 << a.o_rank) : 8;
  for (int j = tid; j < NT; j += 256) colO[j] = lin_bits((uint64_t)(tn * NT + j), a.nO, a.nN) * uO;
  if (tid == 0) abort_flag = 0;
  float sa, sb;
  int ea, eb;
  operand_scale(meta, a.a_meta, hdr, &sa, &ea);
  operand_scale(meta, a.b_meta, hdr, &sb, &eb);
  if (blockIdx.x == 0 && tid == 0)
    meta[a.o_meta].exp = ea + eb + (a.a_meta >= 0 ? meta[a.a_meta].exp : 0) + (a.b_meta >= 0 ? meta[a.b_meta].exp : 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      // the N side's bulk copy (one arrival with its bytes) and 128 converters
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[i])), "r"(1 + TC_M));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_done)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tbase;
  const uint32_t s0 = smem_u32(tsm);
  const int64_t kc = a.kc;
  if (warp == 0) {
    if (lane == 0) {
      const char *srcB = ws + a.pn_off + (sidx * a.ntiles + tn) * kc * BBYTES;
      for (int64_t k = 0; k < kc; ++k) {
        const int st = (int)(k % S);
        if (k >= S && !tc_wait(smem_u32(&bar_empty[st]), (uint32_t)((k / S) - 1) & 1u)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int *)&abort_flag) break;
        const uint32_t fb = smem_u32(&bar_full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(BBYTES) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                s0 + st * SBYTES + ABYTES),
            "l"(srcB + k * BBYTES), "r"(BBYTES), "r"(fb)
            : "memory");
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t fmt = P == 4 ? 0u : 1u;
      constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                 ((uint32_t)(TC_M >> 4) << 24);
      constexpr uint32_t idesc_neg = idesc | (1u << 13);
      for (int64_t k = 0; k < kc; ++k) {
        const int st = (int)(k % S);
        if (!tc_wait(smem_u32(&bar_full[st]), (uint32_t)(k / S) & 1u)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sA = s0 + st * SBYTES, sB = sA + ABYTES;
        uint32_t acc = k > 0 ? 1u : 0u;
        if (P == 4) {
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int i = t == 2 ? 1 : 0, j = t == 1 ? 1 : 0;
            const uint64_t ar = tc_desc(sA + i * tc_plane_bytes(TC_M)), ai = tc_desc(sA + (2 + i) * tc_plane_bytes(TC_M));
            const uint64_t br = tc_desc(sB + j * tc_plane_bytes(NT)), bi = tc_desc(sB + (2 + j) * tc_plane_bytes(NT));
            tc_mma(tmem, ar, br, idesc, acc);
            tc_mma(tmem, ai, bi, idesc_neg, 1u);
            tc_mma(tmem + NT, ar, bi, idesc, acc);
            tc_mma(tmem + NT, ai, br, idesc, 1u);
            acc = 1u;
          }
        } else {
#pragma unroll
          for (int t = 0; t < 6; ++t) {
            const int i = t == 2 || t == 4 ? 1 : t == 5 ? 2 : 0;
            const int j = t == 1 || t == 4 ? 1 : t == 3 ? 2 : 0;
            const uint64_t ar = tc_desc(sA + i * tc_plane_bytes(TC_M)), ai = tc_desc(sA + (3 + i) * tc_plane_bytes(TC_M));
            const uint64_t br = tc_desc(sB + j * tc_plane_bytes(NT)), bi = tc_desc(sB + (3 + j) * tc_plane_bytes(NT));
            tc_mma(tmem, ar, br, idesc, acc);
            tc_mma(tmem, ai, bi, idesc_neg, 1u);
            tc_mma(tmem + NT, ar, bi, idesc, acc);
            tc_mma(tmem + NT, ai, br, idesc, 1u);
            acc = 1u;
          }
        }
        tc_commit(smem_u32(&bar_empty[st]));
      }
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  } else if (warp >= 4) {
    // converters: row r of the M tile.  The raw ring holds, per stage, the
    // 16 complex64 values of each row for one chunk (128 bytes per row, its
    // 16-byte pieces rotated by r mod 8 so a quarter-warp's reads hit
    // distinct banks); each thread fills its own row with 8-byte cp.async
    // copies RS - 1 chunks ahead, so only its own copy groups are waited on.
    const int r = tid - 128;
    const int64_t rho = tm * TC_M + r;
    const bool live = rho < a.mrows;
    const int64_t m = a.fold ? rho / a.Bp : rho, beta = a.fold ? rho % a.Bp : 0;
    const int64_t uA = a.a_batched && !a.a_bout ? (int64_t)a.Bp * 8 : 8;
    const int64_t bstrideA = a.a_bout ? ((int64_t)8 << a.a_rank) : 8;
    const char *rowA = ws + a.a_src_off +
                       (lin_bits((uint64_t)sidx, a.sA, a.ns) + lin_bits((uint64_t)(live ? m : 0), a.mA, a.nM)) * uA +
                       (a.a_batched ? beta * bstrideA : 0);
    const float sc = P == 4 ? sa * 32768.f : sa;
    const int klow = a.nk < 4 ? a.nk : 4;  // summed variables inside a chunk of 16
    const int64_t K = (int64_t)1 << a.nk;
    int64_t klo[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) klo[q] = q < (1 << klow) ? lin_bits((uint64_t)q, a.kA, klow) * uA : 0;
    uint8_t *raw = tsm + S * SBYTES + r * 128;
    const uint32_t raw_s = smem_u32(raw);
    const int rot = r & 7;
    auto issue = [&](int64_t k) {
      const int rs = (int)(k % RS);
      const char *h = rowA + lin_bits((uint64_t)(k * 16), a.kA, a.nk) * uA;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int slot = rs * TC_M * 128 + (((q >> 1) ^ rot) << 4) + ((q & 1) << 3);
        if (live && q < K) {
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(raw_s + slot), "l"(h + klo[q]) : "memory");
        } else {
          *reinterpret_cast<float2 *>(raw + slot) = make_float2(0.f, 0.f);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int64_t k = 0; k < RS - 1; ++k) {
      if (k < kc) issue(k);
      else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int64_t k = 0; k < kc; ++k) {
      if (k + RS - 1 < kc) issue(k + RS - 1);
      else asm volatile("cp.async.commit_group;" ::: "memory");
      // every group but the newest RS - 1 has landed: chunk k's row is in
      asm volatile("cp.async.wait_group %0;" ::"n"(RS - 1) : "memory");
      const int rs = (int)(k % RS);
      float2 v[16];
#pragma unroll
      for (int q2 = 0; q2 < 8; ++q2) {
        const float4 w = *reinterpret_cast<const float4 *>(raw + rs * TC_M * 128 + ((q2 ^ rot) << 4));
        v[2 * q2] = make_float2(w.x * sc, w.y * sc);
        v[2 * q2 + 1] = make_float2(w.z * sc, w.w * sc);
      }
      const int st = (int)(k % S);
      if (k >= S && !tc_wait(smem_u32(&bar_empty[st]), (uint32_t)((k / S) - 1) & 1u)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      conv_put<P>(tsm + st * SBYTES, r, v);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_full[st])) : "memory");
    }
    // no copy of this thread is left in flight when the CTA ends
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  // epilogue: warps 4-7, thread tid - 128 = tile row = tensor-memory lane
  bool ok = tc_wait(smem_u32(&bar_done), 0u);
  if (!ok) ok = tc_wait(smem_u32(&bar_done), 0u);
  ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
  const bool valid_run = ok && !*(volatile int *)&abort_flag;
  float lmax = 0.f;
  if (ok && warp >= 4) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int64_t rho = tm * TC_M + (tid - 128);
    const bool valid = valid_run && rho < a.mrows;
    int64_t m = rho, b2 = 0;
    if (a.fold) {
      m = rho / a.Bp;
      b2 = rho % a.Bp;
    }
    char *orow = ws + a.o_off +
                 (lin_bits((uint64_t)sidx, a.sO, a.ns) + lin_bits((uint64_t)(valid ? m : 0), a.mO, a.nM)) * uO +
                 (a.o_bat ? b2 * bstrideO : 0);
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t re[16], im[16];
      tc_ld16(tl + c0, re);
      tc_ld16(tl + NT + c0, im);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float2 v = make_float2(__uint_as_float(re[j]) * a.out_scale, __uint_as_float(im[j]) * a.out_scale);
          *reinterpret_cast<float2 *>(orow + colO[c0 + j]) = v;
          lmax = fmax_nan(lmax, absmax2(v));
        }
      }
    }
  }
  if (!valid_run && tid == 0 && hdr) atomicCAS(&hdr->status, 0, QGM_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
  record_max(lmax, meta, a.o_meta);
}

// out[x] += F[x] * 2^exp * c in FP64 (one slice's partial amplitudes), then
// advance the slice counter.
__global__ void k_accumulate(const char *ws, int64_t final_off, int final_meta, int final_batched,
                             int open_mode, int64_t n_out, double2 *out, const Meta *meta,
                             Header *hdr, double c_re, double c_im, int rows_log, int Bp) {
  const float2 *F = reinterpret_cast<const float2 *>(ws + final_off);
  const int e = final_meta >= 0 ? meta[final_meta].exp : 0;
  if (final_meta >= 0 && blockIdx.x == 0 && threadIdx.x == 0 &&
      ((meta[final_meta].maxbits >> 23) & 0xff) == 0xff)
    atomicCAS(&hdr->status, 0, QGM_ERR_NONFINITE);
  const double s = ldexp(1.0, e);
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_out;
       x += (int64_t)gridDim.x * blockDim.x) {
    // open outputs: x is the row of the final tensor; a batch: x is the
    // batch entry of its single row (a final tensor without a batch axis is
    // the same for every entry); a batch with open outputs: x = b * 2^k + row
    int64_t src;
    if (open_mode == 1) src = x;
    else if (open_mode == 2)
      src = final_batched ? (x & ((1ll << rows_log) - 1)) * Bp + (x >> rows_log) : (x & ((1ll << rows_log) - 1));
    else src = final_batched ? x : 0;
    const float2 v = F[src];
    const double re = (double)v.x * s, im = (double)v.y * s;
    double2 o = out[x];
    o.x += re * c_re - im * c_im;
    o.y += re * c_im + im * c_re;
    out[x] = o;
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    __threadfence();
    hdr->slice_id += 1;
  }
}

// The final tensor of batch entry 0 as it stands (its exponent left apart),
// times the constant c, in FP64: out[r] for the 2^rows_log open entries.
__global__ void k_raw_final(const char *ws, int64_t final_off, int final_batched, int rows_log, int Bp,
                            double c_re, double c_im, double2 *out, const Meta *meta, int final_meta,
                            int64_t *exp_out) {
  const float2 *F = reinterpret_cast<const float2 *>(ws + final_off);
  const int64_t rows = (int64_t)1 << rows_log;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = F[final_batched ? r * Bp : r];
    out[r] = make_double2((double)v.x * c_re - (double)v.y * c_im, (double)v.x * c_im + (double)v.y * c_re);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *exp_out = final_meta >= 0 ? (int64_t)meta[final_meta].exp : 0;
}

// Adjoint seed: d(final)/d(final) = 1 for every batch entry, exponent 0.
__global__ void k_seed(float2 *seed, int Bp, Meta *meta, int slot) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Bp; t += gridDim.x * blockDim.x)
    seed[t] = make_float2(1.f, 0.f);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    meta[slot].maxbits = __float_as_uint(1.f);
    meta[slot].exp = 0;
  }
}

// dL/dp for one parameter per block (blockIdx.x = 2 gate + which):
// 2 Re( c * 2^E * sum_b conj(g_b) sum_r adj[r][b] D_p[r, x_b] ), with adj the
// adjoint of the gate's leaf (exponent E), D_p its derivative table and
// g_b = dL/d conj(a_b); accumulated in FP64.
__global__ void k_grad_reduce(const char *ws, const GradParam *gp, const uint64_t *bits, int64_t B,
                              int Bp, const double2 *g, const Meta *meta, double c_re, double c_im,
                              double *grad, int slice, int accumulate) {
  __shared__ double red_r[256], red_i[256];
  const int pidx = blockIdx.x >> 1, which = blockIdx.x & 1;
  const GradParam P = gp[pidx];
  const float2 *adj = reinterpret_cast<const float2 *>(ws + P.adj_off);
  const float2 *db = reinterpret_cast<const float2 *>(ws + P.dbase_off[which]);
  const int64_t rows = (int64_t)1 << P.n_int;
  // this slice's values of the leaf's sliced variables (between its
  // internal and output variables in the table index)
  int sbits = 0;
  for (int a = 0; a < P.n_slice; ++a) sbits |= ((slice >> P.slice_bit[a]) & 1) << (P.n_slice - 1 - a);
  double sr = 0.0, si = 0.0;
  for (int64_t t = threadIdx.x; t < rows * B; t += blockDim.x) {
    const int64_t r = t / B, b = t - r * B;
    const float2 a = adj[r * Bp + b];
    int ob = 0;
    if (P.n_out > 0) {
      const uint64_t x = bits[b];
      for (int q = 0; q < P.n_out; ++q) ob |= (int)((x >> P.out_qubit[q]) & 1ull) << (P.n_out - 1 - q);
    }
    const float2 d = db[(((r << P.n_slice) | sbits) << P.n_out) | ob];
    const double xr = (double)a.x * d.x - (double)a.y * d.y;
    const double xi = (double)a.x * d.y + (double)a.y * d.x;
    const double2 gb = g[b];
    sr += gb.x * xr + gb.y * xi;
    si += gb.x * xi - gb.y * xr;
  }
  red_r[threadIdx.x] = sr;
  red_i[threadIdx.x] = si;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      red_r[threadIdx.x] += red_r[threadIdx.x + h];
      red_i[threadIdx.x] += red_i[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sc = ldexp(1.0, meta[P.adj_meta].exp);
    const double Sr = red_r[0] * sc, Si = red_i[0] * sc;
    const double v = 2.0 * (c_re * Sr - c_im * Si);
    grad[blockIdx.x] = accumulate ? grad[blockIdx.x] + v : v;
  }
}

// ---------------------------------------------------------------------------
// Cross-entropy statistics (App. B): FP64 sums of log p, N p and (N p)^2 over
// the amplitudes, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_xeb(const double2 *a, int64_t B, double N, double *sums) {
  __shared__ double r0[1024], r1[1024], r2[1024];
  double s0 = 0, s1 = 0, s2 = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
    const double p = a[b].x * a[b].x + a[b].y * a[b].y;
    s0 += log(p);
    s1 += N * p;
    s2 += (N * p) * (N * p);
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      r0[threadIdx.x] += r0[threadIdx.x + h];
      r1[threadIdx.x] += r1[threadIdx.x + h];
      r2[threadIdx.x] += r2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[0] = r0[0];
    sums[1] = r1[0];
    sums[2] = r2[0];
  }
}

// Cumulative sums of p_j = |a_j|^2 (one block: each thread sums a contiguous
// chunk, a block scan of the chunk totals, then each chunk is written out).
__global__ void __launch_bounds__(1024) k_cumsum_p(const double2 *a, int64_t t, double *cdf) {
  __shared__ double part[1024];
  const int64_t chunk = (t + blockDim.x - 1) / blockDim.x;
  const int64_t lo = threadIdx.x * chunk, hi = lo + chunk < t ? lo + chunk : t;
  double s = 0;
  for (int64_t j = lo; j < hi; ++j) s += a[j].x * a[j].x + a[j].y * a[j].y;
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < (int)blockDim.x; ++i) part[i] += part[i - 1];
  __syncthreads();
  double run = threadIdx.x ? part[threadIdx.x - 1] : 0.0;
  for (int64_t j = lo; j < hi; ++j) {
    run += a[j].x * a[j].x + a[j].y * a[j].y;
    cdf[j] = run;
  }
}

// Draw i: u = the i-th output of SplitMix64(seed) (counter form: the state
// after i + 1 golden-ratio increments, then the two mixing rounds), top 53
// bits; index = first j with cdf[j] / total > u.
__global__ void k_sample(const double *cdf, int64_t t, int64_t m, uint64_t seed, int64_t *idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    const double total = cdf[t - 1];
    int64_t lo = 0, hi = t - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cdf[mid] / total > u) hi = mid;
      else lo = mid + 1;
    }
    idx[i] = lo;
  }
}

// FP32 peak microbenchmark: independent FMA chains per thread (enough of
// them to cover the FMA latency), the result kept live through a sink.
constexpr int FMA_CHAINS = 8;
__device__ float g_fma_sink;
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float x) {
  float acc[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) acc[c] = x + (float)(threadIdx.x + c);
  const float m = 0.999999f, a = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) acc[c] = fmaf(acc[c], m, a);
  }
  float t = 0.f;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) t += acc[c];
  if (t == 12345.678f) g_fma_sink = t;
}

// Zero the FP64 result and the status, restart at slice 0.
__global__ void k_init(double2 *out, int64_t n_out, Header *hdr) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_out;
       x += (int64_t)gridDim.x * blockDim.x)
    out[x] = make_double2(0.0, 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) hdr->slice_id = 0;
}

// ------------------------------------------------------------------------
// Resident executor: one CTA per chunk of Bc bitstrings runs every step of
// the plan with all of its tensors in shared memory; the only global reads
// are the bitstrings and the unbatched gate tables (L1-resident), the only
// global write is the chunk's FP64 amplitudes.  Steps are separated by
// __syncthreads only: no grid-wide barrier, no launch per step.
constexpr int RES_THREADS = 256;

// Product of the M inputs at one term; with PER_LOAD each value is scaled as
// it is loaded, otherwise the caller applies one combined scale per entry.
template <int M, bool PER_LOAD>
__device__ __forceinline__ float2 res_term(const char *sm, const int *rowb, const int *eb,
                                           const float *scale) {
  float2 p = *reinterpret_cast<const float2 *>(sm + rowb[0] + eb[0]);
  if (PER_LOAD) p = make_float2(p.x * scale[0], p.y * scale[0]);
#pragma unroll
  for (int i = 1; i < M; ++i) {
    float2 v = *reinterpret_cast<const float2 *>(sm + rowb[i] + eb[i]);
    if (PER_LOAD) v = make_float2(v.x * scale[i], v.y * scale[i]);
    p = cmul(p, v);
  }
  return p;
}

// One elimination step run by a group of G threads (gt = index in the
// group).  Each input index is linear in the bits of (row, e): a thread
// starts from its first item and term and then only adds the planner's
// table entries selected by the trailing zeros of its item and term counters.
// When the inputs' scale exponents sum to a representable power of two the
// raw product is scaled once per entry (no input's raw values can overflow:
// each stored tensor is a sum of at most 2^8 products of values below 1).
template <int M, bool PER_LOAD>
__device__ __forceinline__ float res_step_body(const RStep &S, char *sm, const float *scale, float comb,
                                               int lb, int lg, int items, int gt, int G) {
  const int k = S.k;
  const int tpi = 1 << lg;
  const int sit = G >> lg;                  // item stride of one thread (>= 2^lb)
  int rowb[M], eb0[M];
  const int it0 = gt >> lg, g = gt & (tpi - 1);
  const uint32_t row0 = (uint32_t)it0 >> lb;
  const uint32_t beta = (uint32_t)it0 & ((1u << lb) - 1u);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const RIn &in = S.in[i];
    int ri = in.soff + (in.batched ? (int)beta * 8 : 0);
    for (int b = 0; b < in.nlow; ++b)
      if ((row0 >> b) & 1u) ri += in.lrow[b];
    rowb[i] = ri;
    int ei = 0;
    for (int b = 0; b < lg; ++b)
      if ((g >> b) & 1) ei += in.lterm[b];
    eb0[i] = ei;
  }
  const int n_iter = (items * tpi + G - 1) / G;
  const int tcount = 1 << (k - lg);
  float lmax = 0.f;
  float2 *o = reinterpret_cast<float2 *>(sm + S.out_soff);
  for (int j = 0; j < n_iter; ++j) {
    const int it = it0 + j * sit;
    const bool live = it < items;
    if (j) {
      const int t = __ffs(j) - 1;
#pragma unroll
      for (int i = 0; i < M; ++i) rowb[i] += S.in[i].rinc[t];
    }
    float2 acc = make_float2(0.f, 0.f);
    if (live) {
      int eb[M];
#pragma unroll
      for (int i = 0; i < M; ++i) eb[i] = eb0[i];
      if (tcount == 1) {
        acc = res_term<M, PER_LOAD>(sm, rowb, eb, scale);
      } else {
        // two terms per iteration: counter values jt (even) and jt + 1
        // differ in bit 0 only (increment tinc[0]); from jt + 1 to jt + 2
        // the carry lands on bit ffs(jt + 2) - 1
        float2 acc2 = make_float2(0.f, 0.f);
        for (int jt = 0; jt < tcount; jt += 2) {
          if (jt) {
            const int t = __ffs(jt) - 1;
#pragma unroll
            for (int i = 0; i < M; ++i) eb[i] += S.in[i].tinc[t];
          }
          int eb2[M];
#pragma unroll
          for (int i = 0; i < M; ++i) eb2[i] = eb[i] + S.in[i].tinc[0];
          const float2 p1 = res_term<M, PER_LOAD>(sm, rowb, eb, scale);
          const float2 p2 = res_term<M, PER_LOAD>(sm, rowb, eb2, scale);
          acc.x += p1.x;
          acc.y += p1.y;
          acc2.x += p2.x;
          acc2.y += p2.y;
          #pragma unroll
          for (int i = 0; i < M; ++i) eb[i] = eb2[i];
        }
        acc.x += acc2.x;
        acc.y += acc2.y;
      }
      if (!PER_LOAD) acc = make_float2(acc.x * comb, acc.y * comb);
    }
    // reduce the tpi partial sums of an item (aligned lane groups; tpi > 1
    // only when every lane runs exactly one iteration)
    for (int q = 1; q < tpi; q <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, q);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, q);
    }
    if (live && g == 0) {
      o[it] = acc;
      lmax = fmax_nan(lmax, absmax2(acc));
    }
  }
  return lmax;
}

template <int M>
__device__ __forceinline__ float res_step(const RStep &S, char *sm, const Meta *meta, Header *hdr,
                                          int logBc, int lb, int lg, int items, int gt, int G,
                                          int *esum_out) {
  (void)logBc;
  float scale[M];
  int esum = 0, es = 0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const RIn &in = S.in[i];
    int e;
    operand_scale(meta, in.meta, hdr, &scale[i], &e);
    es += e;
    esum += e + (in.meta >= 0 ? meta[in.meta].exp : 0);
  }
  *esum_out = esum;
  if (es >= -120 && es <= 120) {
    const float comb = __int_as_float((127 - es) << 23);
    return res_step_body<M, false>(S, sm, scale, comb, lb, lg, items, gt, G);
  }
  return res_step_body<M, true>(S, sm, scale, 1.f, lb, lg, items, gt, G);
}

// The whole pass for one chunk of Bc bitstrings.  Steps come in dependency
// levels; each warp walks its own list of (step, level) entries, runs the
// steps assigned to it with no block barrier inside a level, and every warp
// closes each level with the same __syncthreads.

__global__ void __launch_bounds__(RES_THREADS, 5)
    k_resident(const char *ws, const RStep *steps, const RJob *jobs, int n_jobs, const uint32_t *wlist_g,
               int n_wl, const int32_t *wstart_g, int n_levels, int wlist_soff, const uint64_t *bits,
               int64_t B, int logBc, int n_meta, int final_soff, int final_meta, int final_batched,
               double c_re, double c_im, double2 *out, Header *hdr) {
  extern __shared__ __align__(16) char sm[];
  __shared__ RStep wsd[RES_WARPS];
  const int Bc = 1 << logBc;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t b0 = (int64_t)blockIdx.x * Bc;
  Meta *meta = reinterpret_cast<Meta *>(sm);
  uint32_t *wl = reinterpret_cast<uint32_t *>(sm + wlist_soff);
  for (int i = tid; i < n_meta; i += RES_THREADS) {
    meta[i].maxbits = 0;
    meta[i].exp = 0;
  }
  for (int i = tid; i < n_wl; i += RES_THREADS) wl[i] = __ldg(wlist_g + i);
  const int e0 = __ldg(wstart_g + wid), e1 = __ldg(wstart_g + wid + 1);
  // leaves of this chunk, one job per leaf row: batched rows take the base
  // entry selected by the output bits of x_beta, unbatched rows the entry
  const float2 *wsf = reinterpret_cast<const float2 *>(ws);
  for (int t = tid; t < (n_jobs << logBc); t += RES_THREADS) {
    const int b = t & (Bc - 1);
    const RJob j = jobs[t >> logBc];
    if (!j.batched && b) continue;
    int ob = 0;
    if (j.n_out) {
      const uint64_t x = (b0 + b < B) ? bits[b0 + b] : 0ull;
      ob = j.n_out == 1 ? (int)((x >> j.q0) & 1ull)
                        : (int)((((x >> j.q0) & 1ull) << 1) | ((x >> j.q1) & 1ull));
    }
    reinterpret_cast<float2 *>(sm + j.dst)[j.batched ? b : 0] = __ldg(wsf + j.src + ob);
  }
  __syncthreads();
  RStep &S = wsd[wid];
  int e = e0;
  for (int L = 0; L < n_levels; ++L) {
    while (e < e1 && (int)((wl[e] >> 12) & 0x3ffu) == L) {
      const uint32_t entry = wl[e];
      const int words = (int)(entry >> 22);
      int *dst = reinterpret_cast<int *>(&S);
      const int *src = reinterpret_cast<const int *>(steps + (entry & 0xfffu));
      for (int idx = lane; idx < words; idx += 32) dst[idx] = __ldg(src + idx);
      __syncwarp();
      ++e;
      const int w0 = S.sched & 15, nw = (S.sched >> 4) & 15, lg = (S.sched >> 8) & 15;
      const int lb = S.batched_out ? logBc : 0;
      const int items = (1 << S.w_out) << lb;
      const int gt = tid - 32 * w0, G = 32 * nw;
      float lmax;
      int esum = 0;
      switch (S.m) {
        case 1: lmax = res_step<1>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        case 2: lmax = res_step<2>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        case 3: lmax = res_step<3>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        case 4: lmax = res_step<4>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        case 5: lmax = res_step<5>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        case 6: lmax = res_step<6>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        case 7: lmax = res_step<7>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
        default: lmax = res_step<8>(S, sm, meta, hdr, logBc, lb, lg, items, gt, G, &esum); break;
      }
      for (int q = 16; q > 0; q >>= 1) lmax = fmax_nan(lmax, __shfl_xor_sync(0xffffffffu, lmax, q));
      if (lane == 0) {
        if (lmax > 0.f || lmax != lmax) atomicMax(&meta[S.out_meta].maxbits, __float_as_uint(lmax));
        if (wid == w0) meta[S.out_meta].exp = esum;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  if (tid == 0 && ((meta[final_meta].maxbits >> 23) & 0xff) == 0xff) atomicCAS(&hdr->status, 0, QGM_ERR_NONFINITE);
  if (tid < Bc && b0 + tid < B) {
    const float2 v = reinterpret_cast<const float2 *>(sm + final_soff)[final_batched ? tid : 0];
    const double sc = ldexp(1.0, meta[final_meta].exp);
    const double re = (double)v.x * sc, im = (double)v.y * sc;
    out[b0 + tid] = make_double2(re * c_re - im * c_im, re * c_im + im * c_re);
  }
}

}  // namespace

namespace qgm {
bool jit_kernel(const std::string &src, const std::string &name, int device, cudaKernel_t *out,
                std::string *err);
}

struct qgm_exec_state {
  int device = -1;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  cudaGraphExec_t graph = nullptr;
  const void *g_bits = nullptr;
  void *g_out = nullptr;
  int64_t g_B = -1;
  int sms = 148;
  int kind = QGM_EXEC_STEPWISE;
  int layout = -1;  // index into qgm_plan::resident
  cudaGraphExec_t ggraph = nullptr;  // the adjoint pass, for one set of pointers
  const void *gg_bits = nullptr, *gg_dl = nullptr;
  void *gg_grad = nullptr, *gg_amp = nullptr;
  int64_t gg_B = -1;
  cudaKernel_t jit = nullptr;  // compiled resident kernel (QGM_EXEC_COMPILED)
  cudaKernel_t jit_pre = nullptr;  // its bitstring-independent part, when split off
  std::string jit_error;       // why the compiled kernel is not used, if so
};

static int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return QGM_ERR_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

extern "C" void qgm_exec_release(qgm_plan *p) {
  if (!p || !p->exec) return;
  if (p->exec->graph) cudaGraphExecDestroy(p->exec->graph);
  if (p->exec->ggraph) cudaGraphExecDestroy(p->exec->ggraph);
  delete p->exec;
  p->exec = nullptr;
}

static void launch_leaves(qgm_plan *p, const uint64_t *d_bits, int64_t B, cudaStream_t st) {
  char *ws = p->exec->ws;
  const int nl = (int)p->leafdesc.size();
  k_build_leaves<<<std::max(nl, 1), 256, 0, st>>>(
      ws, reinterpret_cast<const LeafDesc *>(ws + p->off_leafdesc), nl,
      reinterpret_cast<Meta *>(ws + p->off_meta), p->n_meta,
      reinterpret_cast<Header *>(ws + p->off_header), d_bits, B, p->Bp);
}

// Grid of one product-sum step: row strides are powers of two so that the
// kernels can walk rows by table increments.
// Tensor-core form of a GEMM-shaped step: split both operands into planes,
// then the product (see k_split and k_gemm_tc).
static void launch_gemm_tc(char *ws, int sms, int Bp, GemmDesc g, const TcCfg &c, int64_t planes_off, int P,
                           Meta *meta, Header *hdr, cudaStream_t st, cudaEvent_t mid = nullptr, bool conv = false) {
  if (c.swap) gemm_swap_roles(g);
  // a folded step may convert its M side inside the product kernel (then
  // only the N side is split)
  conv = conv && c.fold;
  const int64_t pn_off = planes_off + c.bytesM;
  for (int side = conv ? 1 : 0; side < 2; ++side) {
    const bool ms = side == 0;
    SplitArgs s{};
    s.src_off = ms ? g.a_off : g.b_off;
    s.dst_off = ms ? planes_off : pn_off;
    s.meta = ms ? g.a_meta : g.b_meta;
    s.batched = ms ? g.a_bat : g.b_bat;
    s.fold = ms && c.fold;
    s.perbeta = c.perbeta;
    s.Bp = Bp;
    s.nr = ms ? g.nm : g.nn;
    s.nk = g.nk;
    s.ns = g.ns;
    s.tr = ms ? TC_M : c.nt;
    s.rows = ms ? c.mrows : ((int64_t)1 << g.nn);
    s.rtiles = ms ? c.mtiles : c.ntiles;
    s.kc = c.kc;
    s.fp16 = P == 4;
    s.bout = ms ? g.a_bout : g.b_bout;
    s.rank = (ms ? g.nm : g.nn) + g.nk + g.ns;
    std::memcpy(s.rX, ms ? g.mA : g.nB, GMAXB);
    std::memcpy(s.kX, ms ? g.kA : g.kB, GMAXB);
    std::memcpy(s.sX, ms ? g.sA : g.sB, GMAXB);
    const int64_t items = c.inst * s.rtiles * s.tr * c.kc * 2;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)sms * 16));
    if (P == 4) k_split<4><<<blocks, 256, 0, st>>>(ws, s, meta, hdr);
    else k_split<6><<<blocks, 256, 0, st>>>(ws, s, meta, hdr);
  }
  if (mid) cudaEventRecord(mid, st);
  TcArgs a{};
  a.pm_off = planes_off;
  a.pn_off = pn_off;
  a.o_off = g.o_off;
  a.a_meta = g.a_meta;
  a.b_meta = g.b_meta;
  a.o_meta = g.o_meta;
  a.o_bat = g.o_bat;
  a.fold = c.fold;
  a.perbeta = c.perbeta;
  a.Bp = Bp;
  a.o_bout = g.o_bout;
  // a shared variable among the output's two lowest index bits (one 32-byte
  // sector of complex64) when no batch axis lies below them: instances fastest
  a.s_fast = 0;
  if (g.ns > 0 && !(g.o_bat && !g.o_bout))
    for (int b = 0; b < g.ns; ++b)
      if (g.sO[b] < 2) a.s_fast = 1;
  a.o_rank = g.nm + g.nn + g.ns;
  a.nM = g.nm;
  a.nN = g.nn;
  a.ns = g.ns;
  a.mrows = c.mrows;
  a.mtiles = c.mtiles;
  a.ntiles = c.ntiles;
  a.kc = c.kc;
  a.out_scale = P == 4 ? 0x1p-30f : 1.f;
  std::memcpy(a.mO, g.mO, GMAXB);
  std::memcpy(a.nO, g.nO, GMAXB);
  std::memcpy(a.sO, g.sO, GMAXB);
  a.a_src_off = g.a_off;
  a.a_batched = g.a_bat;
  a.a_bout = g.a_bout;
  a.a_rank = g.nm + g.nk + g.ns;
  a.nk = g.nk;
  std::memcpy(a.mA, g.mA, GMAXB);
  std::memcpy(a.kA, g.kA, GMAXB);
  std::memcpy(a.sA, g.sA, GMAXB);
  const unsigned grid = (unsigned)(c.inst * c.mtiles * c.ntiles);
  if (conv) {
#define QGM_TC_CONV(NT_, P_) \
  k_gemm_tc_conv<NT_, P_><<<grid, 256, tcc_smem_bytes(NT_, P_), st>>>(ws, a, meta, hdr)
    if (P == 4) {
      if (c.nt == 256) QGM_TC_CONV(256, 4);
      else if (c.nt == 128) QGM_TC_CONV(128, 4);
      else if (c.nt == 64) QGM_TC_CONV(64, 4);
      else QGM_TC_CONV(32, 4);
    } else {
      if (c.nt == 256) QGM_TC_CONV(256, 6);
      else if (c.nt == 128) QGM_TC_CONV(128, 6);
      else if (c.nt == 64) QGM_TC_CONV(64, 6);
      else QGM_TC_CONV(32, 6);
    }
#undef QGM_TC_CONV
    return;
  }
#define QGM_TC_LAUNCH(NT_, P_) \
  k_gemm_tc<NT_, P_><<<grid, 128, tc_smem_bytes(NT_, P_), st>>>(ws, a, meta, hdr)
  if (P == 4) {
    if (c.nt == 256) QGM_TC_LAUNCH(256, 4);
    else if (c.nt == 128) QGM_TC_LAUNCH(128, 4);
    else if (c.nt == 64) QGM_TC_LAUNCH(64, 4);
    else QGM_TC_LAUNCH(32, 4);
  } else {
    if (c.nt == 256) QGM_TC_LAUNCH(256, 6);
    else if (c.nt == 128) QGM_TC_LAUNCH(128, 6);
    else if (c.nt == 64) QGM_TC_LAUNCH(64, 6);
    else QGM_TC_LAUNCH(32, 6);
  }
#undef QGM_TC_LAUNCH
}

// Raise the dynamic shared-memory limit of every tensor-core kernel.
static cudaError_t tc_set_smem() {
  cudaError_t e = cudaSuccess;
#define QGM_TC_ATTR(NT_, P_)                                                                                  \
  if (e == cudaSuccess)                                                                                       \
  e = cudaFuncSetAttribute(k_gemm_tc<NT_, P_>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes(NT_, P_))
  QGM_TC_ATTR(256, 4);
  QGM_TC_ATTR(128, 4);
  QGM_TC_ATTR(64, 4);
  QGM_TC_ATTR(32, 4);
  QGM_TC_ATTR(256, 6);
  QGM_TC_ATTR(128, 6);
  QGM_TC_ATTR(64, 6);
  QGM_TC_ATTR(32, 6);
#undef QGM_TC_ATTR
#define QGM_TC_ATTR(NT_, P_)                                                                                  \
  if (e == cudaSuccess)                                                                                       \
  e = cudaFuncSetAttribute(k_gemm_tc_conv<NT_, P_>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                           tcc_smem_bytes(NT_, P_))
  QGM_TC_ATTR(256, 4);
  QGM_TC_ATTR(128, 4);
  QGM_TC_ATTR(64, 4);
  QGM_TC_ATTR(32, 4);
  QGM_TC_ATTR(256, 6);
  QGM_TC_ATTR(128, 6);
  QGM_TC_ATTR(64, 6);
  QGM_TC_ATTR(32, 6);
#undef QGM_TC_ATTR
  return e;
}

static void launch_step_ws(char *ws, int sms, int Bp, const StepDesc &d, const GemmDesc *gemms, Meta *meta,
                           Header *hdr, cudaStream_t st, bool tc = false, int64_t planes_off = 0,
                           int planes = 4, cudaEvent_t mid = nullptr, const StepTune *tn = nullptr) {
  const uint64_t rows = 1ull << d.w_out;
  const bool as_ps = tn && tn->ps;  // a GEMM-shaped step the tuner runs as a product-sum
  if (d.gemm >= 0 && gemms && tc && !as_ps) {
    const TcCfg c = tc_config(gemms[d.gemm], Bp, planes, tn && tn->nt_cap ? tn->nt_cap : 256);
    if (c.ok) {
      launch_gemm_tc(ws, sms, Bp, gemms[d.gemm], c, planes_off, planes, meta, hdr, st, mid, tn && tn->conv);
      return;
    }
  }
  if (d.gemm >= 0 && gemms && gemm_fp32_ok(gemms[d.gemm]) && !as_ps) {
    const GemmDesc &g = gemms[d.gemm];
    const dim3 grid(1u << ((g.nm - 6) + (g.nn - (g.nn >= 6 ? 6 : 5))), g.o_bat ? Bp : 1, 1u << g.ns);
    if (g.nn >= 6) {
      if (g.nk >= 5) k_gemm<32, 64><<<grid, 256, 0, st>>>(ws, g, meta, hdr, Bp);
      else k_gemm<16, 64><<<grid, 256, 0, st>>>(ws, g, meta, hdr, Bp);
    } else {
      if (g.nk >= 5) k_gemm<32, 32><<<grid, 256, 0, st>>>(ws, g, meta, hdr, Bp);
      else k_gemm<16, 32><<<grid, 256, 0, st>>>(ws, g, meta, hdr, Bp);
    }
    return;
  }
  auto pow2_floor = [](uint64_t v) {
    uint64_t r = 1;
    while (r * 2 <= v) r *= 2;
    return r;
  };
  if (d.batched_out) {
    const int pairs = Bp / 2;
    int logP = -1;  // narrow batch: 2^logP pair slots per row, 128 / 2^logP rows per block
    if (pairs <= 64) {
      logP = 0;
      while ((1 << logP) < pairs) ++logP;
    }
    const int bx = logP < 0 ? (pairs + STEP_THREADS - 1) / STEP_THREADS : 1;
    const uint64_t rpb = logP < 0 ? 1 : (uint64_t)(STEP_THREADS >> logP);
    const uint64_t row_blocks = (rows + rpb - 1) / rpb;
    const uint64_t cap = (uint64_t)std::max(1, sms * 16 / bx);
    // split the summed terms over threadIdx.y while the grid is small
    int T = 1;
    while (T < 4 && (T * 2) <= (1 << std::min(d.k, 4)) &&
           row_blocks * (uint64_t)bx * STEP_THREADS * T < (uint64_t)sms * 1024)
      T *= 2;
    if (tn && tn->T > 0 && tn->T <= 4 && tn->T <= (1 << std::min(d.k, 4))) T = tn->T;
    if (d.tile_t > 0) {
      // rows are counted over the output bits outside the tile
      const uint64_t orows = rows >> d.tile_t;
      const uint64_t oblocks = (orows + rpb - 1) / rpb;
      const uint64_t gy = pow2_floor(std::min<uint64_t>(oblocks, std::min<uint64_t>(cap, 32768)));
      const dim3 gt(bx, (unsigned)gy);
      switch (d.m) {
        case 1: k_step_tile<1><<<gt, STEP_THREADS, 0, st>>>(ws, d, meta, hdr, Bp, logP); break;
        case 2: k_step_tile<2><<<gt, STEP_THREADS, 0, st>>>(ws, d, meta, hdr, Bp, logP); break;
        case 3: k_step_tile<3><<<gt, STEP_THREADS, 0, st>>>(ws, d, meta, hdr, Bp, logP); break;
        case 4: k_step_tile<4><<<gt, STEP_THREADS, 0, st>>>(ws, d, meta, hdr, Bp, logP); break;
        default: k_step_tile<MAXIN><<<gt, STEP_THREADS, 0, st>>>(ws, d, meta, hdr, Bp, logP); break;
      }
      return;
    }
    const uint64_t gy = pow2_floor(std::min<uint64_t>(row_blocks, std::min<uint64_t>(cap, 32768)));
    const dim3 g2(bx, (unsigned)gy), b2(STEP_THREADS, T);
    // four or eight terms in flight per thread where the tuner measured that
    // faster (each thread's term count 2^(k - log2 T) must hold them)
    const int tbits = d.k - (31 - __builtin_clz((unsigned)T));
    const int uu = tn && tn->U == 8 && tbits >= 3 ? 8 : (tn && tn->U >= 4 && tbits >= 2 ? 4 : 2);
#define QGM_SB(M_)                                                                      \
  if (uu == 8) k_step_batched<M_, 8><<<g2, b2, 0, st>>>(ws, d, meta, hdr, Bp, logP);    \
  else if (uu == 4) k_step_batched<M_, 4><<<g2, b2, 0, st>>>(ws, d, meta, hdr, Bp, logP); \
  else k_step_batched<M_, 2><<<g2, b2, 0, st>>>(ws, d, meta, hdr, Bp, logP);
    switch (d.m) {
      case 1: QGM_SB(1) break;
      case 2: QGM_SB(2) break;
      case 3: QGM_SB(3) break;
      case 4: QGM_SB(4) break;
      case 5: QGM_SB(5) break;
      case 6: QGM_SB(6) break;
      case 7: QGM_SB(7) break;
      default: QGM_SB(8) break;
    }
#undef QGM_SB
  } else {
    const uint64_t blocks = pow2_floor(std::max<uint64_t>(1, std::min<uint64_t>((rows + 255) / 256, (uint64_t)sms * 8)));
    switch (d.m) {
      case 1: k_step_plain<1><<<(unsigned)blocks, 256, 0, st>>>(ws, d, meta, hdr); break;
      case 2: k_step_plain<2><<<(unsigned)blocks, 256, 0, st>>>(ws, d, meta, hdr); break;
      case 3: k_step_plain<3><<<(unsigned)blocks, 256, 0, st>>>(ws, d, meta, hdr); break;
      case 4: k_step_plain<4><<<(unsigned)blocks, 256, 0, st>>>(ws, d, meta, hdr); break;
      default: k_step_plain<MAXIN><<<(unsigned)blocks, 256, 0, st>>>(ws, d, meta, hdr); break;
    }
  }
}

// The autotuner's parameters of a forward step (none for the adjoint steps).
static const StepTune *tune_of(const qgm_plan *p, const StepDesc &d) {
  if (p->steps.empty() || &d < p->steps.data() || &d >= p->steps.data() + p->steps.size()) return nullptr;
  const size_t i = (size_t)(&d - p->steps.data());
  return i < p->tune.size() ? &p->tune[i] : nullptr;
}

static void launch_step(qgm_plan *p, const StepDesc &d, cudaStream_t st, cudaEvent_t mid = nullptr) {
  char *ws = p->exec->ws;
  launch_step_ws(ws, p->exec->sms, p->Bp, d, p->gemms.data(), reinterpret_cast<Meta *>(ws + p->off_meta),
                 reinterpret_cast<Header *>(ws + p->off_header), st, p->gemm_tc, p->off_planes, p->tc_planes, mid,
                 tune_of(p, d));
}

// Autotuner (qgm_plan_opts.autotune; candidates: the tensor-core N tile, for
// folded steps in-kernel conversion of the M side, the product-sum term
// groups): one pass over an all-zero batch puts
// real tensors in the workspace; then, step by step in order, every
// candidate launch configuration of a step with several is run once to
// warm up and three times under CUDA events, and the fastest is kept (the
// candidates compute the same products; only a term split changes the
// order of a sum).  Steps whose fixed-rule launch takes under 0.05 ms are
// left alone.  Ends with the status word cleared.
static int autotune(qgm_plan *p, cudaStream_t st) {
  qgm_exec_state *x = p->exec;
  uint64_t *d_bits = reinterpret_cast<uint64_t *>(x->ws + p->off_bits);
  CK(cudaMemsetAsync(d_bits, 0, (size_t)p->Bp * 8, st));
  launch_leaves(p, d_bits, p->batch, st);
  for (const StepDesc &d : p->steps) launch_step(p, d, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_step = [&](const StepDesc &d, float *ms) -> int {
    launch_step(p, d, st);
    CK(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) launch_step(p, d, st);
    CK(cudaEventRecord(e1, st));
    CK(cudaGetLastError());
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= 3.f;
    return QGM_OK;
  };
  for (size_t si = 0; si < p->steps.size(); ++si) {
    const StepDesc &d = p->steps[si];
    StepTune &tn = p->tune[si];
    std::vector<StepTune> cand;
    if (d.gemm >= 0 && p->gemm_tc && tc_config(p->gemms[d.gemm], p->Bp, p->tc_planes).ok) {
      const TcCfg tcc = tc_config(p->gemms[d.gemm], p->Bp, p->tc_planes);
      for (int conv = 0; conv <= (tcc.fold ? 1 : 0); ++conv)
        for (int cap : {256, 128, 64})
          if (cap <= tcc.nt) {
            StepTune t;
            t.nt_cap = cap;
            t.conv = conv;
            cand.push_back(t);
          }
    }
    if (d.gemm >= 0 && d.batched_out && d.tile_t == 0) {
      // a GEMM-shaped step may also run as a product-sum (batch axis
      // innermost everywhere: coalesced across batch entries)
      const GemmDesc &g = p->gemms[d.gemm];
      if (!g.a_bout && !g.b_bout && !g.o_bout)
        for (int U : {2, 4}) {
          StepTune t;
          t.ps = 1;
          t.U = U;
          cand.push_back(t);
        }
    } else if (d.gemm < 0 && d.batched_out && d.tile_t == 0) {
      for (int U : {2, 4, 8})
        for (int T : {1, 2, 4})
          if (T <= (1 << std::min(d.k, 4)) && (U == 2 || (1 << d.k) >= U * T)) {
            StepTune t;
            t.T = T;
            t.U = U;
            cand.push_back(t);
          }
    }
    if (cand.size() < 2) continue;
    float ms_rule = 0.f;
    StepTune rule{};
    rule.conv = p->opts.tc_convert ? 1 : 0;
    tn = rule;
    int rc = time_step(d, &ms_rule);
    if (rc) return rc;
    if (ms_rule < 0.05f) continue;
    StepTune best = rule;
    float best_ms = ms_rule;
    for (const StepTune &c : cand) {
      tn = c;
      float ms = 0.f;
      rc = time_step(d, &ms);
      if (rc) return rc;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    tn = best;
    tn.ms_rule = ms_rule;
    tn.ms_best = best_ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaMemsetAsync(x->ws + p->off_header, 0, sizeof(int32_t), st));
  CK(cudaStreamSynchronize(st));
  return QGM_OK;
}

static void launch_accumulate(qgm_plan *p, double2 *d_out, int64_t n_out, cudaStream_t st) {
  char *ws = p->exec->ws;
  const int64_t blocks = std::min<int64_t>((n_out + 255) / 256, (int64_t)p->exec->sms * 8);
  // the fixed-gate tables had 2^{-1/2} pulled out half_pow_total times
  const cd c = p->constant * std::pow(2.0, -0.5 * p->half_pow_total);
  k_accumulate<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
      ws, p->final_off, p->final_meta, p->final_batched,
      p->output_mode == QGM_OUT_OPEN ? 1 : (p->open_in_batch ? 2 : 0), n_out, d_out,
      reinterpret_cast<const Meta *>(ws + p->off_meta), reinterpret_cast<Header *>(ws + p->off_header), c.real(),
      c.imag(), p->open_in_batch, p->Bp);
}

// Enqueue one slice: leaves, steps, accumulation.
static int enqueue_slice(qgm_plan *p, const uint64_t *d_bits, int64_t B, double2 *d_out,
                         int64_t n_out, cudaStream_t st) {
  launch_leaves(p, d_bits, B, st);
  char *ws = p->exec->ws;
  for (size_t s = 0; s < p->steps.size();) {
    const int32_t g = s < p->plain_group.size() ? p->plain_group[s] : 0;
    if (g >= 2) {
      // a run of small batch-free steps: one launch of one CTA
      k_step_plain_group<<<1, 256, 0, st>>>(ws, reinterpret_cast<const StepDesc *>(ws + p->off_sdesc), (int)s, g,
                                            reinterpret_cast<Meta *>(ws + p->off_meta),
                                            reinterpret_cast<Header *>(ws + p->off_header));
      s += (size_t)g;
    } else {
      launch_step(p, p->steps[s], st);
      ++s;
    }
  }
  launch_accumulate(p, d_out, n_out, st);
  return QGM_OK;
}

static void launch_resident(qgm_plan *p, const uint64_t *d_bits, int64_t B, double2 *d_out,
                            cudaStream_t st) {
  qgm_exec_state *x = p->exec;
  const ResidentLayout &L = p->resident[x->layout];
  const int logBc = __builtin_ctz(L.chunk);
  const int64_t G = (B + L.chunk - 1) / L.chunk;
  const cd c = p->constant * std::pow(2.0, -0.5 * p->half_pow_total);
  const char *ws = x->ws;
  const char *rs = ws + p->off_rsteps;
  const RJob *jobs = reinterpret_cast<const RJob *>(rs + L.steps.size() * sizeof(RStep));
  const uint32_t *wl = reinterpret_cast<const uint32_t *>(rs + L.steps.size() * sizeof(RStep) +
                                                          L.jobs.size() * sizeof(RJob));
  const int32_t *wst = reinterpret_cast<const int32_t *>(wl + L.wlist.size());
  if (x->kind == QGM_EXEC_COMPILED) {
    const char *ws_c = ws;
    int n_jobs = (int)L.jobs.size();
    long long Bl = (long long)B;
    double cr = c.real(), ci = c.imag();
    Header *hdr = reinterpret_cast<Header *>(x->ws + p->off_header);
    void *args[] = {&ws_c, &jobs, &n_jobs, &d_bits, &Bl, &cr, &ci, &d_out, &hdr};
    const size_t smem = (size_t)compiled_smem(L);
    if (!x->jit_pre) {
      cudaLaunchKernel(reinterpret_cast<const void *>(x->jit), dim3((unsigned)G), dim3(RES_THREADS), args, smem, st);
      return;
    }
    // the bitstring-independent part once (one CTA), then the batched part;
    // the latter may start early and waits for the former's outputs
    cudaLaunchKernel(reinterpret_cast<const void *>(x->jit_pre), dim3(1), dim3(RES_THREADS), args, smem, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(RES_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(x->jit), args);
    return;
  }
  k_resident<<<(unsigned)G, RES_THREADS, (size_t)L.smem_bytes, st>>>(
      ws, reinterpret_cast<const RStep *>(rs), jobs, (int)L.jobs.size(), wl, (int)L.wlist.size(), wst,
      L.n_levels, L.wlist_soff, d_bits, B, logBc, p->n_meta_fwd, L.final_soff, L.final_meta, p->final_batched,
      c.real(), c.imag(), d_out, reinterpret_cast<Header *>(x->ws + p->off_header));
}

static int run(qgm_plan *p, const uint64_t *d_bits, int64_t B, double2 *d_out, int64_t n_out,
               cudaStream_t st) {
  qgm_exec_state *x = p->exec;
  if (x->kind == QGM_EXEC_RESIDENT || x->kind == QGM_EXEC_COMPILED) {
    launch_resident(p, d_bits, B, d_out, st);
    CK(cudaGetLastError());
    return QGM_OK;
  }
  Header *hdr = reinterpret_cast<Header *>(x->ws + p->off_header);
  const int64_t nslices = (int64_t)1 << p->slice_vars.size();
  if (!x->graph || x->g_bits != d_bits || x->g_out != d_out || x->g_B != B) {
    if (x->graph) {
      cudaGraphExecDestroy(x->graph);
      x->graph = nullptr;
    }
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_slice(p, d_bits, B, d_out, n_out, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&x->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    x->g_bits = d_bits;
    x->g_out = d_out;
    x->g_B = B;
  }
  const int64_t iblocks = std::min<int64_t>((n_out + 255) / 256, (int64_t)x->sms * 4);
  k_init<<<(unsigned)std::max<int64_t>(iblocks, 1), 256, 0, st>>>(d_out, n_out, hdr);
  CK(cudaGetLastError());
  for (int64_t s = 0; s < nslices; ++s) CK(cudaGraphLaunch(x->graph, st));
  return QGM_OK;
}

static int check_bound(qgm_plan *p, const char *fn) {
  if (!p) {
    set_error("%s: null plan", fn);
    return QGM_ERR_ARG;
  }
  if (!p->exec || !p->exec->ws) {
    set_error("%s: no workspace bound (call qgm_plan_bind first)", fn);
    return QGM_ERR_ARG;
  }
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != p->exec->device) {
    set_error("%s: current device %d differs from the bound device %d", fn, dev, p->exec->device);
    return QGM_ERR_ARG;
  }
  return QGM_OK;
}

// Initial shared memory of the compiled resident kernel: zeros (tensor
// metadata included) with the bitstring-independent leaf rows in place and
// the recorded maxima of the steps with a static bound (2^k, exponent 0).
static int upload_image(qgm_plan *p, const ResidentLayout &L, int smem, cudaStream_t st) {
  const int64_t shift = worklist_bytes(L);
  std::vector<float> img((size_t)smem / 4, 0.f);
  for (const RJob &j : L.jobs) {
    if (j.batched) continue;
    const int64_t d = (j.dst - shift) / 4, s2 = 2 * (int64_t)j.src - p->off_base / 4;
    img[d] = p->base_tables[s2];
    img[d + 1] = p->base_tables[s2 + 1];
  }
  for (const auto &sb : static_bounds(L)) {
    const uint32_t bits = (uint32_t)(127 + sb.second.first) << 23;
    const int32_t ex = sb.second.second;
    std::memcpy(&img[2 * (size_t)sb.first], &bits, 4);
    std::memcpy(&img[2 * (size_t)sb.first + 1], &ex, 4);
  }
  CK(cudaMemcpyAsync(p->exec->ws + p->off_image, img.data(), img.size() * 4, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return QGM_OK;
}

// Self-test of the bounded wait (qgm_selftest_wait_timeout): one mbarrier
// with an arrival count of 1; with arrive = 0 nothing arrives, so the wait
// for its first phase runs out after limit_ns and the kernel writes
// QGM_ERR_TIMEOUT; with arrive = 1 the thread arrives first and the wait
// succeeds at once.
__device__ int32_t g_selftest_status;
__global__ void k_selftest_wait(uint64_t limit_ns, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    g_selftest_status = tc_wait_ns(smem_u32(&bar), 0u, limit_ns) ? QGM_OK : QGM_ERR_TIMEOUT;
  }
}

extern "C" {

int qgm_plan_bind(qgm_plan *p, void *d_workspace, size_t ws_bytes, void *stream) {
  if (!p || !d_workspace) {
    set_error("qgm_plan_bind: null argument");
    return QGM_ERR_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    set_error("qgm_plan_bind: no CUDA device");
    return QGM_ERR_NOGPU;
  }
  if (((uintptr_t)d_workspace & 255) != 0) {
    set_error("qgm_plan_bind: workspace must be 256-byte aligned");
    return QGM_ERR_ARG;
  }
  if ((int64_t)ws_bytes < p->ws_bytes) {
    set_error("qgm_plan_bind: workspace of %zu bytes, the plan needs %lld", ws_bytes,
              (long long)p->ws_bytes);
    return QGM_ERR_OOM;
  }
  qgm_exec_release(p);
  p->exec = new qgm_exec_state;
  qgm_exec_state *x = p->exec;
  CK(cudaGetDevice(&x->device));
  CK(cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, x->device));
  x->ws = static_cast<char *>(d_workspace);
  if (p->gemm_tc && !p->gemms.empty()) CK(tc_set_smem());
  x->ws_bytes = ws_bytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(x->ws + p->off_header, 0, 256, st));
  if (!p->base_tables.empty())
    CK(cudaMemcpyAsync(x->ws + p->off_base, p->base_tables.data(), p->base_tables.size() * sizeof(float),
                       cudaMemcpyHostToDevice, st));
  if (!p->leafdesc.empty())
    CK(cudaMemcpyAsync(x->ws + p->off_leafdesc, p->leafdesc.data(), p->leafdesc.size() * sizeof(LeafDesc),
                       cudaMemcpyHostToDevice, st));
  if (!p->steps.empty())
    CK(cudaMemcpyAsync(x->ws + p->off_sdesc, p->steps.data(), p->steps.size() * sizeof(StepDesc),
                       cudaMemcpyHostToDevice, st));
  if (p->grad && !p->gparams.empty())
    CK(cudaMemcpyAsync(x->ws + p->off_gparams, p->gparams.data(), p->gparams.size() * sizeof(GradParam),
                       cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  // executor: compiled resident, else resident, when a layout fits; the
  // chunk size by fewest waves x chunk
  x->kind = QGM_EXEC_STEPWISE;
  x->layout = -1;
  for (StepTune &t : p->tune) {
    t = StepTune{};
    t.conv = p->opts.tc_convert ? 1 : 0;
  }
  if (p->executor_pref == QGM_EXEC_STEPWISE || p->resident.empty()) {
    if (p->executor_pref == QGM_EXEC_RESIDENT || p->executor_pref == QGM_EXEC_COMPILED) {
      set_error("qgm_plan_bind: this plan has no resident layout (one slice, batch outputs only)");
      return QGM_ERR_ARG;
    }
    if (p->opts.autotune && p->output_mode == QGM_OUT_BATCH) return autotune(p, st);
    return QGM_OK;
  }
  int optin = 0, sm_smem = 0, reserved = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, x->device));
  CK(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, x->device));
  CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, x->device));
  auto waves_x_chunk = [&](const ResidentLayout &L, int cps) {
    const int64_t G = (p->batch + L.chunk - 1) / L.chunk;
    return (double)((G + (int64_t)x->sms * cps - 1) / ((int64_t)x->sms * cps)) * L.chunk;
  };
  auto upload = [&](const ResidentLayout &L) -> int {
    CK(cudaMemcpyAsync(x->ws + p->off_rsteps, L.steps.data(), L.steps.size() * sizeof(RStep),
                       cudaMemcpyHostToDevice, st));
    char *rs = x->ws + p->off_rsteps;
    const size_t jo = L.steps.size() * sizeof(RStep), wo = jo + L.jobs.size() * sizeof(RJob);
    if (!L.jobs.empty())
      CK(cudaMemcpyAsync(rs + jo, L.jobs.data(), L.jobs.size() * sizeof(RJob), cudaMemcpyHostToDevice, st));
    if (!L.wlist.empty())
      CK(cudaMemcpyAsync(rs + wo, L.wlist.data(), L.wlist.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(rs + wo + L.wlist.size() * 4, L.wstart, sizeof(L.wstart), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return QGM_OK;
  };
  if (p->executor_pref == QGM_EXEC_AUTO || p->executor_pref == QGM_EXEC_COMPILED) {
    // the pass as a kernel generated for this plan: as many CTAs per SM as
    // shared memory allows (at most 8), registers bounded to match
    int best_li = -1, best_cps = 0;
    double best = -1;
    for (size_t li = 0; li < p->resident.size(); ++li) {
      const ResidentLayout &L = p->resident[li];
      if (p->opts.resident_chunk > 0 && L.chunk != p->opts.resident_chunk) continue;
      const int64_t smem = compiled_smem(L);
      if (smem > optin) continue;
      const int cps = (int)std::min<int64_t>(8, sm_smem / (smem + reserved));
      if (cps < 1) continue;
      const double cost = waves_x_chunk(L, cps);
      if (best < 0 || cost < best) {
        best = cost;
        best_li = (int)li;
        best_cps = cps;
      }
    }
    if (best_li >= 0) {
      const ResidentLayout &L = p->resident[best_li];
      const int smem = (int)compiled_smem(L);
      // the bitstring-independent steps run once per call in a kernel of
      // their own when the batch takes two or more waves of CTAs (in one
      // wave that kernel's latency outweighs what each CTA saves)
      const bool split = L.split_pre && waves_x_chunk(L, best_cps) >= 2.0 * L.chunk;
      cudaKernel_t k = nullptr, kp = nullptr;
      bool ok = jit_kernel(resident_source(p, L, "qgm_resident_plan", best_cps, split ? RES_MAIN : RES_WHOLE),
                           "qgm_resident_plan", x->device, &k, &x->jit_error);
      if (ok && split)
        ok = jit_kernel(resident_source(p, L, "qgm_resident_pre", 1, RES_PRE), "qgm_resident_pre", x->device, &kp,
                        &x->jit_error);
      if (ok) {
        CK(cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem, x->device));
        if (kp) CK(cudaKernelSetAttributeForDevice(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem, x->device));
        int rc = upload(L);
        if (rc) return rc;
        rc = upload_image(p, L, smem, st);
        if (rc) return rc;
        x->jit = k;
        x->jit_pre = kp;
        x->layout = best_li;
        x->kind = QGM_EXEC_COMPILED;
        return QGM_OK;
      }
    } else {
      x->jit_error = "no layout fits the device's shared memory";
    }
    if (p->executor_pref == QGM_EXEC_COMPILED) {
      set_error("qgm_plan_bind: compiled resident kernel unavailable: %s", x->jit_error.c_str());
      return QGM_ERR_ARG;
    }
  }
  double best = -1;
  for (size_t li = 0; li < p->resident.size(); ++li) {
    const ResidentLayout &L = p->resident[li];
    if (p->opts.resident_chunk > 0 && L.chunk != p->opts.resident_chunk) continue;
    if (L.smem_bytes + (int64_t)sizeof(RStep) + 64 > optin) continue;
    CK(cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes));
    int cps = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, k_resident, RES_THREADS, (size_t)L.smem_bytes));
    if (cps < 1) continue;
    const double cost = waves_x_chunk(L, cps);
    if (best < 0 || cost < best) {
      best = cost;
      x->layout = (int)li;
    }
  }
  if (x->layout >= 0) {
    const ResidentLayout &L = p->resident[x->layout];
    CK(cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes));
    int rc = upload(L);
    if (rc) return rc;
    x->kind = QGM_EXEC_RESIDENT;
  } else if (p->executor_pref == QGM_EXEC_RESIDENT) {
    set_error("qgm_plan_bind: no resident layout fits this device's shared memory");
    return QGM_ERR_ARG;
  }
  if (x->kind == QGM_EXEC_STEPWISE && p->opts.autotune && p->output_mode == QGM_OUT_BATCH) return autotune(p, st);
  return QGM_OK;
}

int qgm_plan_set_params(qgm_plan *p, const double *params, int64_t n, void *stream) {
  if (!p || (!params && n > 0)) {
    set_error("qgm_plan_set_params: null argument");
    return QGM_ERR_ARG;
  }
  if (n != 2 * (int64_t)p->model.param_factor.size()) {
    set_error("qgm_plan_set_params: %lld values for %zu parameters", (long long)n, 2 * p->model.param_factor.size());
    return QGM_ERR_ARG;
  }
  int rc = plan_set_params(p, params);
  if (rc) return rc;
  if (!p->exec || !p->exec->ws) return QGM_OK;  // uploaded at bind
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!p->base_tables.empty())
    CK(cudaMemcpyAsync(p->exec->ws + p->off_base, p->base_tables.data(), p->base_tables.size() * sizeof(float),
                       cudaMemcpyHostToDevice, st));
  if (p->exec->kind == QGM_EXEC_COMPILED) {
    const ResidentLayout &L = p->resident[p->exec->layout];
    return upload_image(p, L, (int)compiled_smem(L), st);
  }
  CK(cudaStreamSynchronize(st));
  return QGM_OK;
}

int qgm_plan_get_executor(const qgm_plan *p, int32_t *kind, int32_t *chunk, int64_t *smem_bytes) {
  if (!p || !p->exec) {
    set_error("qgm_plan_get_executor: plan not bound");
    return QGM_ERR_ARG;
  }
  const qgm_exec_state *x = p->exec;
  if (kind) *kind = x->kind;
  const bool res = x->kind == QGM_EXEC_RESIDENT || x->kind == QGM_EXEC_COMPILED;
  if (chunk) *chunk = res ? p->resident[x->layout].chunk : (int32_t)p->Bp;
  if (smem_bytes)
    *smem_bytes = !res ? 0
                       : x->kind == QGM_EXEC_COMPILED ? compiled_smem(p->resident[x->layout])
                                                      : p->resident[x->layout].smem_bytes;
  return QGM_OK;
}

int qgm_amplitudes(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out, void *stream) {
  int rc = check_bound(p, "qgm_amplitudes");
  if (rc) return rc;
  if (p->output_mode != QGM_OUT_BATCH) {
    set_error("qgm_amplitudes: plan has open outputs (use qgm_eliminate)");
    return QGM_ERR_ARG;
  }
  if (B < 1 || B > p->batch || !d_bitstrings || !d_out) {
    set_error("qgm_amplitudes: need 1 <= B <= %lld and non-null buffers", (long long)p->batch);
    return QGM_ERR_ARG;
  }
  return run(p, d_bitstrings, B, reinterpret_cast<double2 *>(d_out), B << p->open_in_batch,
             static_cast<cudaStream_t>(stream));
}

int qgm_amplitudes_host(qgm_plan *p, const uint64_t *h_bitstrings, int64_t B, double *h_out,
                        void *stream) {
  int rc = check_bound(p, "qgm_amplitudes_host");
  if (rc) return rc;
  if (p->output_mode != QGM_OUT_BATCH || B < 1 || B > p->batch || !h_bitstrings || !h_out) {
    set_error("qgm_amplitudes_host: need a batch plan, 1 <= B <= %lld and non-null buffers",
              (long long)p->batch);
    return QGM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Page-locked host buffers the device can address (registered or pinned
  // memory has a device pointer): the resident executors, which read each
  // bitstring once and write each amplitude once, use them in place.
  if ((p->exec->kind == QGM_EXEC_RESIDENT || p->exec->kind == QGM_EXEC_COMPILED) && p->open_in_batch == 0) {
    cudaPointerAttributes ab{}, ao{};
    const bool mapped = cudaPointerGetAttributes(&ab, h_bitstrings) == cudaSuccess &&
                        ab.type == cudaMemoryTypeHost && ab.devicePointer != nullptr &&
                        cudaPointerGetAttributes(&ao, h_out) == cudaSuccess && ao.type == cudaMemoryTypeHost &&
                        ao.devicePointer != nullptr;
    cudaGetLastError();  // a query on pageable memory may leave an error behind
    if (mapped) {
      rc = run(p, static_cast<const uint64_t *>(ab.devicePointer), B, static_cast<double2 *>(ao.devicePointer), B,
               st);
      if (rc) return rc;
      CK(cudaStreamSynchronize(st));
      return QGM_OK;
    }
  }
  uint64_t *d_bits = reinterpret_cast<uint64_t *>(p->exec->ws + p->off_bits);
  double2 *d_out = reinterpret_cast<double2 *>(p->exec->ws + p->off_outstage);
  CK(cudaMemcpyAsync(d_bits, h_bitstrings, B * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  rc = run(p, d_bits, B, d_out, B << p->open_in_batch, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h_out, d_out, (B << p->open_in_batch) * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return QGM_OK;
}

int qgm_eliminate(qgm_plan *p, double *d_out, void *stream) {
  int rc = check_bound(p, "qgm_eliminate");
  if (rc) return rc;
  if (p->output_mode != QGM_OUT_OPEN || !d_out) {
    set_error("qgm_eliminate: needs a plan with open outputs and a non-null output");
    return QGM_ERR_ARG;
  }
  uint64_t *d_bits = reinterpret_cast<uint64_t *>(p->exec->ws + p->off_bits);
  return run(p, d_bits, 1, reinterpret_cast<double2 *>(d_out), p->final_entries,
             static_cast<cudaStream_t>(stream));
}

int qgm_eliminate_fixed(qgm_plan *p, const uint8_t *fixed_assign, double *d_out, int64_t *exp_out, void *stream) {
  int rc = check_bound(p, "qgm_eliminate_fixed");
  if (rc) return rc;
  if (p->output_mode != QGM_OUT_BATCH || !fixed_assign || !d_out || !exp_out) {
    set_error("qgm_eliminate_fixed: needs a batch plan and non-null arguments");
    return QGM_ERR_ARG;
  }
  uint64_t x = 0;
  for (int q = 0; q < p->model.n; ++q) {
    if (fixed_assign[q] > 1) {
      set_error("qgm_eliminate_fixed: output value of qubit %d is %d, not 0 or 1", q, (int)fixed_assign[q]);
      return QGM_ERR_ARG;
    }
    x |= (uint64_t)fixed_assign[q] << q;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  qgm_exec_state *xs = p->exec;
  uint64_t *d_bits = reinterpret_cast<uint64_t *>(xs->ws + p->off_bits);
  double2 *out = reinterpret_cast<double2 *>(d_out);
  const int64_t n_out = (int64_t)1 << p->open_in_batch;
  CK(cudaMemcpyAsync(d_bits, &x, sizeof x, cudaMemcpyHostToDevice, st));
  if (!p->slice_vars.empty()) {
    // slices carry exponents of their own: their FP64 sum, exponent 0
    rc = run(p, d_bits, 1, out, n_out, st);
    if (rc) return rc;
    *exp_out = 0;
    CK(cudaStreamSynchronize(st));
    return QGM_OK;
  }
  // the stepwise launches (whatever executor is bound: the final tensor must
  // be in the workspace), then the raw final tensor and its exponent
  Header *hdr = reinterpret_cast<Header *>(xs->ws + p->off_header);
  k_init<<<1, 32, 0, st>>>(out, 0, hdr);
  launch_leaves(p, d_bits, 1, st);
  for (const StepDesc &d : p->steps) launch_step(p, d, st);
  int64_t *d_exp = reinterpret_cast<int64_t *>(xs->ws + p->off_outstage);
  const cd c = p->constant * std::pow(2.0, -0.5 * p->half_pow_total);
  k_raw_final<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n_out + 255) / 256, 1024)), 256, 0, st>>>(
      xs->ws, p->final_off, p->final_batched, p->open_in_batch, p->Bp, c.real(), c.imag(), out,
      reinterpret_cast<const Meta *>(xs->ws + p->off_meta), p->final_meta, d_exp);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(exp_out, d_exp, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return QGM_OK;
}

int qgm_amplitudes_report(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out, qgm_report *rep,
                          void *stream) {
  if (!rep) {
    set_error("qgm_amplitudes_report: null report");
    return QGM_ERR_ARG;
  }
  std::memset(rep, 0, sizeof *rep);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, st));
  int rc = qgm_amplitudes(p, d_bitstrings, B, d_out, stream);
  if (rc) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    rep->status = rc;
    return rc;
  }
  CK(cudaEventRecord(b, st));
  CK(cudaEventSynchronize(b));
  CK(cudaEventElapsedTime(&rep->ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const qgm_exec_state *x = p->exec;
  rep->executor = x->kind;
  rep->slices = (int64_t)1 << p->slice_vars.size();
  rep->bytes = p->sim.bytes * (double)rep->slices;
  rep->flops = p->sim.flops * (double)rep->slices;
  if (x->kind == QGM_EXEC_STEPWISE) {
    // per slice: leaves, accumulation, and per step one launch (a run of
    // small batch-free steps: one for the run), a tensor-core step adding
    // its split passes (one when its streamed operand is converted in the
    // product kernel, else two)
    int64_t per = 2;
    for (size_t si = 0; si < p->steps.size();) {
      const int32_t g = si < p->plain_group.size() ? p->plain_group[si] : 0;
      if (g >= 2) {
        per += 1;
        si += (size_t)g;
        continue;
      }
      const StepDesc &d = p->steps[si];
      const StepTune *tn = si < p->tune.size() ? &p->tune[si] : nullptr;
      per += 1;
      if (d.gemm >= 0 && p->gemm_tc && !(tn && tn->ps)) {
        const TcCfg c = tc_config(p->gemms[d.gemm], p->Bp, p->tc_planes, tn && tn->nt_cap ? tn->nt_cap : 256);
        if (c.ok) per += tn && tn->conv && c.fold ? 1 : 2;
      }
      ++si;
    }
    rep->launches = per * rep->slices + 1;
  } else {
    rep->launches = x->jit_pre ? 2 : 1;
  }
  rep->status = qgm_status(p, stream);
  if (rep->status < 0) {
    set_error("qgm_amplitudes_report: device status %d", rep->status);
    return rep->status;
  }
  return QGM_OK;
}

int qgm_plan_profile(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out, float *ms,
                     void *stream) {
  int rc = check_bound(p, "qgm_plan_profile");
  if (rc) return rc;
  if (p->output_mode != QGM_OUT_BATCH || B < 1 || B > p->batch || !d_bitstrings || !d_out || !ms) {
    set_error("qgm_plan_profile: need a batch plan, 1 <= B <= %lld and non-null buffers",
              (long long)p->batch);
    return QGM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (int)p->steps.size() + 2;
  if (p->exec->kind == QGM_EXEC_RESIDENT || p->exec->kind == QGM_EXEC_COMPILED) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, st));
    launch_resident(p, d_bitstrings, B, reinterpret_cast<double2 *>(d_out), st);
    CK(cudaEventRecord(b, st));
    CK(cudaGetLastError());
    CK(cudaEventSynchronize(b));
    for (int i = 0; i < n; ++i) ms[i] = 0.f;
    CK(cudaEventElapsedTime(&ms[0], a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return QGM_OK;
  }
  std::vector<cudaEvent_t> ev(n + 1);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  Header *hdr = reinterpret_cast<Header *>(p->exec->ws + p->off_header);
  k_init<<<1, 256, 0, st>>>(reinterpret_cast<double2 *>(d_out), B << p->open_in_batch, hdr);
  CK(cudaEventRecord(ev[0], st));
  launch_leaves(p, d_bitstrings, B, st);
  CK(cudaEventRecord(ev[1], st));
  for (size_t s = 0; s < p->steps.size(); ++s) {
    launch_step(p, p->steps[s], st);
    CK(cudaEventRecord(ev[2 + s], st));
  }
  launch_accumulate(p, reinterpret_cast<double2 *>(d_out), B << p->open_in_batch, st);
  CK(cudaEventRecord(ev[n], st));
  CK(cudaGetLastError());
  CK(cudaEventSynchronize(ev[n]));
  for (int i = 0; i < n; ++i) CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
  for (auto &e : ev) cudaEventDestroy(e);
  return QGM_OK;
}

int qgm_plan_profile_gemm(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, double *d_out, float *ms_split,
                          float *ms_product, void *stream) {
  int rc = check_bound(p, "qgm_plan_profile_gemm");
  if (rc) return rc;
  if (p->output_mode != QGM_OUT_BATCH || B < 1 || B > p->batch || !d_bitstrings || !d_out || !ms_split ||
      !ms_product) {
    set_error("qgm_plan_profile_gemm: need a batch plan, 1 <= B <= %lld and non-null buffers",
              (long long)p->batch);
    return QGM_ERR_ARG;
  }
  if (p->exec->kind != QGM_EXEC_STEPWISE) {
    set_error("qgm_plan_profile_gemm: needs the stepwise executor");
    return QGM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Header *hdr = reinterpret_cast<Header *>(p->exec->ws + p->off_header);
  k_init<<<1, 256, 0, st>>>(reinterpret_cast<double2 *>(d_out), B << p->open_in_batch, hdr);
  launch_leaves(p, d_bitstrings, B, st);
  std::vector<cudaEvent_t> ev;
  std::vector<int> n_ev;
  for (const StepDesc &d : p->steps) {
    if (d.gemm < 0) {
      launch_step(p, d, st);
      continue;
    }
    cudaEvent_t e[3];
    for (auto &x : e) CK(cudaEventCreate(&x));
    CK(cudaEventRecord(e[0], st));
    const bool tc = p->gemm_tc && tc_config(p->gemms[d.gemm], p->Bp, p->tc_planes).ok;
    if (!tc) CK(cudaEventRecord(e[1], st));  // no split pass: all of it is the product
    launch_step(p, d, st, tc ? e[1] : nullptr);
    CK(cudaEventRecord(e[2], st));
    for (auto &x : e) ev.push_back(x);
  }
  launch_accumulate(p, reinterpret_cast<double2 *>(d_out), B << p->open_in_batch, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  for (size_t c = 0; c < ev.size() / 3; ++c) {
    CK(cudaEventElapsedTime(&ms_split[c], ev[3 * c], ev[3 * c + 1]));
    CK(cudaEventElapsedTime(&ms_product[c], ev[3 * c + 1], ev[3 * c + 2]));
  }
  for (auto &x : ev) cudaEventDestroy(x);
  return QGM_OK;
}

int qgm_plan_step_stats(qgm_plan *p, uint32_t *maxbits, int32_t *exps, int64_t cap, void *stream) {
  int rc = check_bound(p, "qgm_plan_step_stats");
  if (rc) return rc;
  if (!maxbits || !exps) {
    set_error("qgm_plan_step_stats: null argument");
    return QGM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<Meta> m((size_t)std::max(p->n_meta, 1));
  CK(cudaMemcpyAsync(m.data(), p->exec->ws + p->off_meta, (size_t)p->n_meta * sizeof(Meta), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int64_t s = 0; s < std::min<int64_t>(cap, (int64_t)p->steps.size()); ++s) {
    const int slot = p->steps[s].out_meta;
    maxbits[s] = slot >= 0 && slot < p->n_meta ? m[slot].maxbits : 0u;
    exps[s] = slot >= 0 && slot < p->n_meta ? m[slot].exp : 0;
  }
  return QGM_OK;
}

int qgm_plan_set_tuning(qgm_plan *p, const int32_t *rec, int64_t n) {
  int rc = check_bound(p, "qgm_plan_set_tuning");
  if (rc) return rc;
  if (n < 0 || (n > 0 && !rec)) {
    set_error("qgm_plan_set_tuning: bad record count or null records");
    return QGM_ERR_ARG;
  }
  for (int64_t c = 0; c < n; ++c) {
    const int32_t *r = rec + 6 * c;
    bool ok = r[0] >= 0 && r[0] < (int32_t)p->steps.size() &&
              (r[1] == 0 || r[1] == 64 || r[1] == 128 || r[1] == 256) &&
              (r[2] == 0 || r[2] == 1 || r[2] == 2 || r[2] == 4) && (r[3] == 0 || r[3] == 1) &&
              (r[4] == 0 || r[4] == 2 || r[4] == 4 || r[4] == 8) && (r[5] == 0 || r[5] == 1);
    if (ok && r[5]) {
      // a product-sum needs the batch axis innermost on every tensor of the step
      const StepDesc &d = p->steps[r[0]];
      ok = d.gemm >= 0 && !p->gemms[d.gemm].a_bout && !p->gemms[d.gemm].b_bout && !p->gemms[d.gemm].o_bout;
    }
    if (!ok) {
      set_error("qgm_plan_set_tuning: bad record %lld (step %d, N tile %d, T %d, conv %d, U %d, ps %d)",
                (long long)c, r[0], r[1], r[2], r[3], r[4], r[5]);
      return QGM_ERR_ARG;
    }
  }
  for (int64_t c = 0; c < n; ++c) {
    const int32_t *r = rec + 6 * c;
    StepTune &t = p->tune[r[0]];
    t.nt_cap = r[1];
    t.T = r[2];
    t.conv = r[3];
    t.U = r[4];
    t.ps = r[5];
    t.ms_rule = t.ms_best = 0.f;
  }
  // the captured passes hold the old launch parameters
  qgm_exec_state *x = p->exec;
  if (x->graph) {
    cudaGraphExecDestroy(x->graph);
    x->graph = nullptr;
  }
  if (x->ggraph) {
    cudaGraphExecDestroy(x->ggraph);
    x->ggraph = nullptr;
  }
  return QGM_OK;
}

int qgm_selftest_wait_timeout(int64_t limit_ns, int32_t arrive, int32_t *status_out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!status_out || limit_ns < 1000 || limit_ns > 2000000000ll) {
    set_error("qgm_selftest_wait_timeout: need status_out and 1 us <= limit_ns <= 2 s");
    return QGM_ERR_ARG;
  }
  const int32_t unset = 1;
  CK(cudaMemcpyToSymbolAsync(g_selftest_status, &unset, sizeof(int32_t), 0, cudaMemcpyHostToDevice, st));
  k_selftest_wait<<<1, 32, 0, st>>>((uint64_t)limit_ns, arrive ? 1 : 0);
  CK(cudaGetLastError());
  CK(cudaMemcpyFromSymbolAsync(status_out, g_selftest_status, sizeof(int32_t), 0, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return QGM_OK;
}

int qgm_measure_fp32_peak(double *tflops, void *stream) {
  if (!tflops) {
    set_error("qgm_measure_fp32_peak: null argument");
    return QGM_ERR_ARG;
  }
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int iters = 1 << 14;
  const dim3 grid((unsigned)sms * 8), block(256);
  k_fma_peak<<<grid, block, 0, st>>>(iters, 1.f);  // warm-up
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, st));
  const int reps = 5;
  for (int r = 0; r < reps; ++r) k_fma_peak<<<grid, block, 0, st>>>(iters, 1.f);
  CK(cudaEventRecord(b, st));
  CK(cudaGetLastError());
  CK(cudaEventSynchronize(b));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double flops = (double)reps * grid.x * block.x * (double)iters * FMA_CHAINS * 2.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return QGM_OK;
}

int qgm_xeb_stats(const double *d_amps, int64_t B, int n_qubits, double *d_scratch, qgm_xeb_result *out,
                  void *stream) {
  if (!d_amps || !d_scratch || !out || B < 1 || n_qubits < 1 || n_qubits > 64) {
    set_error("qgm_xeb_stats: bad arguments");
    return QGM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double N = std::ldexp(1.0, n_qubits);
  k_xeb<<<1, 1024, 0, st>>>(reinterpret_cast<const double2 *>(d_amps), B, N, d_scratch);
  CK(cudaGetLastError());
  double h[3];
  CK(cudaMemcpyAsync(h, d_scratch, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double gamma = 0.5772156649015329, logN = n_qubits * std::log(2.0);
  const double S = -h[0] / (double)B;
  out->cross_entropy = S;
  out->alpha = ((logN + gamma) - S) / ((logN + gamma) - (logN - 1 + gamma));
  out->mean_Np = h[1] / (double)B;
  out->second_moment = h[2] / (double)B;
  return QGM_OK;
}

int qgm_sample_from_set(const double *d_amps, int64_t t, int64_t m, uint64_t seed, double *d_scratch,
                        int64_t *d_idx, void *stream) {
  if (!d_amps || !d_scratch || !d_idx || t < 1 || m < 0) {
    set_error("qgm_sample_from_set: bad arguments");
    return QGM_ERR_ARG;
  }
  if (m == 0) return QGM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_cumsum_p<<<1, 1024, 0, st>>>(reinterpret_cast<const double2 *>(d_amps), t, d_scratch);
  const int64_t blocks = std::min<int64_t>((m + 255) / 256, 4096);
  k_sample<<<(unsigned)blocks, 256, 0, st>>>(d_scratch, t, m, seed, d_idx);
  CK(cudaGetLastError());
  return QGM_OK;
}

int qgm_status(qgm_plan *p, void *stream) {
  int rc = check_bound(p, "qgm_status");
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t s = 0;
  CK(cudaMemcpyAsync(&s, p->exec->ws + p->off_header, sizeof s, cudaMemcpyDeviceToHost, st));
  CK(cudaMemsetAsync(p->exec->ws + p->off_header, 0, sizeof s, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

}  // extern "C"
static void enqueue_grad(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, const double *d_dL_dconja,
                         double *d_grad, double2 *amp, cudaStream_t st);
extern "C" {

int qgm_amplitude_grad(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, const double *d_dL_dconja,
                       double *d_grad, double *d_amp, void *stream) {
  int rc = check_bound(p, "qgm_amplitude_grad");
  if (rc) return rc;
  if (!p->grad) {
    set_error("qgm_amplitude_grad: the plan was made without opts.gradients");
    return QGM_ERR_ARG;
  }
  if (B < 1 || B > p->batch || !d_bitstrings || !d_dL_dconja || !d_grad) {
    set_error("qgm_amplitude_grad: need 1 <= B <= %lld and non-null buffers", (long long)p->batch);
    return QGM_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  qgm_exec_state *x = p->exec;
  double2 *amp = d_amp ? reinterpret_cast<double2 *>(d_amp) : reinterpret_cast<double2 *>(x->ws + p->off_outstage);
  // the pass (hundreds of short launches) runs as one CUDA graph, captured
  // on the first call with this set of pointers
  if (!x->ggraph || x->gg_bits != d_bitstrings || x->gg_dl != d_dL_dconja || x->gg_grad != d_grad ||
      x->gg_amp != amp || x->gg_B != B) {
    if (x->ggraph) {
      cudaGraphExecDestroy(x->ggraph);
      x->ggraph = nullptr;
    }
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_grad(p, d_bitstrings, B, d_dL_dconja, d_grad, amp, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture (adjoint)");
    e = cudaGraphInstantiate(&x->ggraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (adjoint)");
    x->gg_bits = d_bitstrings;
    x->gg_dl = d_dL_dconja;
    x->gg_grad = d_grad;
    x->gg_amp = amp;
    x->gg_B = B;
  }
  CK(cudaGraphLaunch(x->ggraph, st));
  return QGM_OK;
}

}  // extern "C"

// Forward elimination keeping every intermediate, FP64 amplitudes, the seed,
// the backward steps and the per-gate reduction (qgm_amplitude_grad).
static void enqueue_grad(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B, const double *d_dL_dconja,
                         double *d_grad, double2 *amp, cudaStream_t st) {
  qgm_exec_state *x = p->exec;
  char *ws = x->ws;
  Header *hdr = reinterpret_cast<Header *>(ws + p->off_header);
  Meta *meta = reinterpret_cast<Meta *>(ws + p->off_meta);
  const int64_t iblocks = std::min<int64_t>((B + 255) / 256, (int64_t)x->sms * 4);
  k_init<<<(unsigned)std::max<int64_t>(iblocks, 1), 256, 0, st>>>(amp, B, hdr);
  const cd c = p->constant * std::pow(2.0, -0.5 * p->half_pow_total);
  const int n_gates = (int)p->gparams.size();
  // a = sum over slices of a_s: per slice the forward intermediates are
  // recomputed (leaves for that slice, every step kept), then the adjoint
  // pass of that slice; the per-gate reduction adds each slice's share
  const int64_t nslices = (int64_t)1 << p->slice_vars.size();
  for (int64_t s = 0; s < nslices; ++s) {
    launch_leaves(p, d_bitstrings, B, st);
    for (const StepDesc &d : p->gfwd) launch_step(p, d, st);
    k_accumulate<<<(unsigned)std::max<int64_t>(iblocks, 1), 256, 0, st>>>(
        ws, p->g_final_off, p->g_final_meta, 1, 0, B, amp, meta, hdr, c.real(), c.imag(), 0, p->Bp);
    k_seed<<<(p->Bp + 255) / 256, 256, 0, st>>>(reinterpret_cast<float2 *>(ws + p->g_seed_off), p->Bp, meta,
                                                 p->g_seed_meta);
    for (const StepDesc &d : p->gbwd) launch_step(p, d, st);
    if (n_gates > 0)
      k_grad_reduce<<<2 * n_gates, 256, 0, st>>>(ws, reinterpret_cast<const GradParam *>(ws + p->off_gparams),
                                                 d_bitstrings, B, p->Bp,
                                                 reinterpret_cast<const double2 *>(d_dL_dconja), meta, c.real(),
                                                 c.imag(), d_grad, (int)s, s > 0 ? 1 : 0);
  }
}

// ===========================================================================
// Allocation-free entry point.
//
// Some callers cannot allocate device memory at the moment they need
// amplitudes: a host framework whose pool allocator owns all device memory
// and forbids side allocations, or a latency-critical loop in which a
// cudaMalloc/cudaFree would synchronise the device.  For them the stepwise
// kernels run with their scratch (the workspace of qgm_plan_bind) in one
// file-scope device array of QGM_STATIC_SCRATCH_BYTES.  Every GPU that loads
// this library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address (it names a
// host-side stand-in), so the first call on each device, with that device
// current, looks the address up with cudaGetSymbolAddress and caches it.
// That first call should therefore come before any stream capture.  Every
// call shares the one array and leaves the previous call's contents in it;
// everything the kernels need zeroed (status, slice counter, tensor maxima,
// the FP64 result) is cleared by the call itself.  Calls whose work overlaps
// on the GPU (different streams, or other host threads) race on the array.
// ===========================================================================
namespace {

static __device__ __align__(256) char g_static_scratch[QGM_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
char *g_static_addr[128] = {nullptr};

int static_scratch_address(int dev, char **out) {
  if (dev < 0 || dev >= 128) {
    set_error("qgm_amplitudes_static: device ordinal %d out of range", dev);
    return QGM_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void *a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_addr[dev] = static_cast<char *>(a);
  }
  *out = g_static_addr[dev];
  return QGM_OK;
}

// The stepwise launches of one slice with an explicit workspace base.
void static_slice(const qgm_plan *p, char *ws, int sms, const uint64_t *d_bits, int64_t B,
                  double2 *d_out, cudaStream_t st) {
  Meta *meta = reinterpret_cast<Meta *>(ws + p->off_meta);
  Header *hdr = reinterpret_cast<Header *>(ws + p->off_header);
  const int nl = (int)p->leafdesc.size();
  k_build_leaves<<<std::max(nl, 1), 256, 0, st>>>(ws, reinterpret_cast<const LeafDesc *>(ws + p->off_leafdesc),
                                                   nl, meta, p->n_meta, hdr, d_bits, B, p->Bp);
  for (const StepDesc &d : p->steps) launch_step_ws(ws, sms, p->Bp, d, p->gemms.data(), meta, hdr, st);
  const int64_t blocks = std::min<int64_t>((B + 255) / 256, (int64_t)sms * 8);
  const cd c = p->constant * std::pow(2.0, -0.5 * p->half_pow_total);
  k_accumulate<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
      ws, p->final_off, p->final_meta, p->final_batched, p->open_in_batch ? 2 : 0, B << p->open_in_batch, d_out,
      meta, hdr, c.real(), c.imag(), p->open_in_batch, p->Bp);
}

}  // namespace

extern "C" int qgm_amplitudes_static(qgm_plan *p, const uint64_t *d_bitstrings, int64_t B,
                                     double *d_out, void *stream) {
  if (!p || !d_bitstrings || !d_out) {
    set_error("qgm_amplitudes_static: null argument");
    return QGM_ERR_ARG;
  }
  if (p->output_mode != QGM_OUT_BATCH || B < 1 || B > p->batch) {
    set_error("qgm_amplitudes_static: needs a batch plan and 1 <= B <= %lld", (long long)p->batch);
    return QGM_ERR_ARG;
  }
  for (const GemmDesc &g : p->gemms)
    if (g.a_bout || g.b_bout || g.o_bout) {
      set_error("qgm_amplitudes_static: the plan keeps batch-outer intermediates for its tensor-core steps "
                "(larger than the static scratch); use qgm_plan_bind");
      return QGM_ERR_OOM;
    }
  if (p->ws_fwd_bytes > (int64_t)QGM_STATIC_SCRATCH_BYTES) {
    set_error("qgm_amplitudes_static: the plan needs %lld bytes of scratch, more than the %llu-byte "
              "static scratch; use qgm_plan_bind with a caller-allocated workspace",
              (long long)p->ws_fwd_bytes, (unsigned long long)QGM_STATIC_SCRATCH_BYTES);
    return QGM_ERR_OOM;
  }
  int dev = -1, sms = 0;
  CK(cudaGetDevice(&dev));
  char *ws = nullptr;
  int rc = static_scratch_address(dev, &ws);
  if (rc) return rc;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the previous call's plan may have left other tables here: reload ours
  CK(cudaMemsetAsync(ws + p->off_header, 0, 256, st));
  if (!p->base_tables.empty())
    CK(cudaMemcpyAsync(ws + p->off_base, p->base_tables.data(), p->base_tables.size() * sizeof(float),
                       cudaMemcpyHostToDevice, st));
  if (!p->leafdesc.empty())
    CK(cudaMemcpyAsync(ws + p->off_leafdesc, p->leafdesc.data(), p->leafdesc.size() * sizeof(LeafDesc),
                       cudaMemcpyHostToDevice, st));
  Header *hdr = reinterpret_cast<Header *>(ws + p->off_header);
  double2 *out = reinterpret_cast<double2 *>(d_out);
  const int64_t iblocks = std::min<int64_t>((B + 255) / 256, (int64_t)sms * 4);
  k_init<<<(unsigned)std::max<int64_t>(iblocks, 1), 256, 0, st>>>(out, B << p->open_in_batch, hdr);
  const int64_t nslices = (int64_t)1 << p->slice_vars.size();
  for (int64_t s = 0; s < nslices; ++s) static_slice(p, ws, sms, d_bitstrings, B, out, st);
  CK(cudaGetLastError());
  return QGM_OK;
}
