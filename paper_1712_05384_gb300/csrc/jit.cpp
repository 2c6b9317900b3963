// Plan-specialised resident kernel (compiled at bind time with NVRTC).
//
// The resident executor runs the whole elimination of one chunk of
// bitstrings inside one CTA (Sec. IV, App. A: every bucket's product-sum
// with all tensors in shared memory).  Its generic form reads a descriptor
// per step (index-map tables, warp schedule) and walks it at run time; for
// the small steps that dominate low-depth circuits that bookkeeping costs
// more than the arithmetic.  This file writes the same computation as CUDA
// source with every plan constant in place (shared-memory offsets, index
// maps, loop bounds, the warp schedule of each dependency level), so that
// each step is only its loads, complex products and stores, and compiles it
// for the device with NVRTC (loaded with dlopen; when it is missing, or the
// compile fails, the generic resident kernel runs instead).
//
// Arithmetic follows the generic kernel: per-tensor power-of-two exponents
// (the producer records max |re|,|im|; the consumer scales by 2^-e), one
// combined scale per output entry when the inputs' exponents sum to a
// representable power of two, the inputs rescaled in place otherwise.  Two
// additions: short chains of steps over gate tables take a static bound as
// their recorded maximum (static_bounds), and shared memory starts from a
// plan image built at bind.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "host.h"

namespace qgm {

namespace {

// Value of union bit b in input i of step d, in float2 elements (0 when the
// input does not hold that variable).
std::vector<int64_t> union_values(const InDesc &in, int U, int64_t unit) {
  std::vector<int64_t> v(U, 0);
  for (int q = 0; q < in.nruns; ++q)
    for (int l = 0; l < in.len[q]; ++l) v[in.src[q] + l] = ((int64_t)1 << (in.dst[q] + l)) * unit;
  return v;
}

// C expression for sum_b bit_b(x) * val[lo + b], b < n, with val[] powers of
// two or 0: runs of consecutive bits whose values double become one
// shift-and-mask term.
std::string bit_map_expr(const std::string &x, const std::vector<int64_t> &val, int lo, int n) {
  std::string e;
  int b = 0;
  while (b < n) {
    if (val[lo + b] == 0) {
      ++b;
      continue;
    }
    int l = 1;
    while (b + l < n && val[lo + b + l] == val[lo + b] * ((int64_t)1 << l)) ++l;
    const int s = __builtin_ctzll((unsigned long long)val[lo + b]);
    std::ostringstream t;
    t << "(((" << x << " >> " << b << ") & " << ((1 << l) - 1) << ") << " << s << ")";
    e += (e.empty() ? "" : " + ") + t.str();
    b += l;
  }
  return e.empty() ? "0" : e;
}

int64_t bit_map_value(int64_t x, const std::vector<int64_t> &val, int lo, int n) {
  int64_t r = 0;
  for (int b = 0; b < n; ++b)
    if ((x >> b) & 1) r += val[lo + b];
  return r;
}

const char *kPrelude = R"(
typedef unsigned long long u64;
struct Header { int status; int slice_id; int pad[62]; };
struct Meta { unsigned maxbits; int exp; };
struct RJob { int src; int dst; unsigned char n_out, q0, q1, batched; };
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a += x * y (complex), as four fused multiply-adds
__device__ __forceinline__ void cmac(float2 &a, float2 x, float2 y) {
  a.x = fmaf(x.x, y.x, a.x);
  a.x = fmaf(-x.y, y.y, a.x);
  a.y = fmaf(x.x, y.y, a.y);
  a.y = fmaf(x.y, y.x, a.y);
}
__device__ __forceinline__ void opscale(const Meta *meta, int slot, float &s, int &e, int &esum) {
  const unsigned bits = meta[slot].maxbits;
  const int E = (int)((bits >> 23) & 0xff);
  s = 1.f;
  e = 0;
  // Inf or NaN (E = 0xff) stays unscaled: it reaches the final tensor,
  // whose check sets the status
  if (E != 0 && E != 0xff) {
    e = E - 126;
    if (e > 126) e = 126;
    s = __int_as_float((127 - e) << 23);
  }
  esum += e + meta[slot].exp;
}
)";

constexpr int kUnroll = 16;  // terms per unrolled block

// "acc += f0 * f1 * ... " for the given operand expressions: products in a
// chain, the last factor fused into the accumulation
void emit_term(std::ostringstream &o, const std::vector<std::string> &f, const std::string &acc,
               const std::string &ind) {
  if (f.size() == 1) {
    o << ind << "{ const float2 p = " << f[0] << "; " << acc << ".x += p.x; " << acc << ".y += p.y; }\n";
    return;
  }
  o << ind << "{ float2 p = " << f[0] << ";\n";
  for (size_t i = 1; i + 1 < f.size(); ++i) o << ind << "  p = cmul(p, " << f[i] << ");\n";
  o << ind << "  cmac(" << acc << ", p, " << f.back() << "); }\n";
}

// One step's body for the threads of its warps (gt = thread index in the
// group): every item's product-sum with raw operand values, times `comb`
// (2^-es, the inputs' combined scale) per entry.  Shared-memory offsets are
// the layout's minus `shift` (the generic kernel's work lists are not kept).
void emit_body(std::ostringstream &o, const qgm_plan *p, const ResidentLayout &L, size_t q, int64_t shift,
               bool track_max) {
  const RStep &r = L.steps[q];
  const StepDesc &d = p->steps[L.src_step[q]];
  const int logBc = __builtin_ctz(L.chunk);
  const int m = d.m, k = d.k, w = d.w_out, U = w + k;
  const int nw = (r.sched >> 4) & 15, lg = (r.sched >> 8) & 15;
  const int lb = r.batched_out ? logBc : 0;
  const int64_t items = ((int64_t)1 << w) << lb;
  const int G = 32 * nw, tpi = 1 << lg, sit = G >> lg;
  const int64_t n_iter = (items * tpi + G - 1) / G;
  const bool always_live = (items * tpi) % G == 0 && items * tpi >= G;
  const int tpt_log = k - lg;  // terms per thread per item: 2^tpt_log
  const int unr_log = std::min(tpt_log, __builtin_ctz(kUnroll));
  const int blk_log = tpt_log - unr_log;
  std::vector<std::vector<int64_t>> v(m);
  for (int i = 0; i < m; ++i) v[i] = union_values(d.in[i], U, r.in[i].batched ? L.chunk : 1);
  const std::string live = always_live ? "true" : "it < " + std::to_string(items);
  // nested evaluation: the lanes of an entry split the outer terms, each
  // lane runs all 2^k2 inner terms per outer term
  const StepRec &st = p->sim.steps[L.src_step[q]];
  const int k2 = st.k_inner, k1 = k - k2;
  const bool nested = k2 > 0 && k2 <= 4 && lg <= k1 && (int)st.inner.size() == m;
  const int glo = nested ? w + k2 : w;  // union bit of the lane index's bit 0
  if (track_max) o << "    unsigned lmax = 0u;\n";
  if (lg) {
    o << "    const int g = gt & " << (tpi - 1) << ";\n";
    for (int i = 0; i < m; ++i) o << "    const int go" << i << " = " << bit_map_expr("g", v[i], glo, lg) << ";\n";
  }
  o << "#pragma unroll 1\n    for (int j = 0; j < " << n_iter << "; ++j) {\n";
  o << "      const int it = (gt >> " << lg << ") + j * " << sit << ";\n";
  o << "      float2 acc = make_float2(0.f, 0.f);\n";
  o << "      if (" << live << ") {\n";
  if (w) o << "        const int row = it >> " << lb << ";\n";
  if (lb) o << "        const int beta = it & " << ((1 << lb) - 1) << ";\n";
  for (int i = 0; i < m; ++i) {
    o << "        const int b" << i << " = " << ((r.in[i].soff - shift) / 8);
    if (r.in[i].batched && lb) o << " + beta";
    o << " + " << bit_map_expr("row", v[i], 0, w);
    if (lg) o << " + go" << i;
    o << ";\n";
  }
  if (nested) {
    // term index e = (e1 << k2) | e2 with e1 = (blk << (u1_log + lg)) | (u1 << lg) | g
    const int u2n = 1 << k2;
    const int u1_log = std::min(k1 - lg, std::max(0, 4 - k2));
    const int blk_log1 = k1 - lg - u1_log;
    o << "        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);\n";
    o << "#pragma unroll 1\n        for (int blk = 0; blk < " << (1 << blk_log1) << "; ++blk) {\n";
    for (int i = 0; i < m; ++i) {
      const std::string e = blk_log1 ? bit_map_expr("blk", v[i], w + k2 + lg + u1_log, blk_log1) : std::string("0");
      o << "          const int c" << i << " = b" << i << " + " << e << ";\n";
    }
    for (int u1 = 0; u1 < (1 << u1_log); ++u1) {
      o << "          { float2 i0 = make_float2(0.f, 0.f), i1 = make_float2(0.f, 0.f);\n";
      for (int u2 = 0; u2 < u2n; ++u2) {
        const int64_t e = ((int64_t)u1 << (lg + k2)) | u2;
        std::vector<std::string> f;
        for (int i = 0; i < m; ++i)
          if (st.inner[i]) f.push_back("F[c" + std::to_string(i) + " + " + std::to_string(bit_map_value(e, v[i], w, k)) + "]");
        emit_term(o, f, "i" + std::to_string(u2 & 1), "            ");
      }
      const int64_t e = (int64_t)u1 << (lg + k2);
      std::vector<std::string> f = {"make_float2(i0.x + i1.x, i0.y + i1.y)"};
      for (int i = 0; i < m; ++i)
        if (!st.inner[i]) f.push_back("F[c" + std::to_string(i) + " + " + std::to_string(bit_map_value(e, v[i], w, k)) + "]");
      emit_term(o, f, "a" + std::to_string(u1 & 1), "            ");
      o << "          }\n";
    }
    o << "        }\n";
  } else {
  // unrolled blocks of 2^unr_log terms: the block's offsets at run time,
  // the term offsets inside a block as constants; term index
  // e = (blk << (unr_log + lg)) | (u << lg) | g
  o << "        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);\n";
  o << "#pragma unroll 1\n        for (int blk = 0; blk < " << (1 << blk_log) << "; ++blk) {\n";
  for (int i = 0; i < m; ++i) {
    const std::string e = blk_log ? bit_map_expr("blk", v[i], w + lg + unr_log, blk_log) : std::string("0");
    o << "          const int c" << i << " = b" << i << " + " << e << ";\n";
  }
  for (int u = 0; u < (1 << unr_log); ++u) {
    std::vector<std::string> f;
    for (int i = 0; i < m; ++i)
      f.push_back("F[c" + std::to_string(i) + " + " + std::to_string(bit_map_value((int64_t)u << lg, v[i], w, k)) + "]");
    emit_term(o, f, "a" + std::to_string(u & 1), "          ");
  }
  o << "        }\n";
  }
  o << "        acc = make_float2((a0.x + a1.x) * comb, (a0.y + a1.y) * comb);\n";
  o << "      }\n";
  for (int s2 = 1; s2 < tpi; s2 <<= 1)
    o << "      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, " << s2
      << "); acc.y += __shfl_xor_sync(0xffffffffu, acc.y, " << s2 << ");\n";
  o << "      if (" << live << (lg ? " && g == 0" : "") << ") {\n";
  o << "        F[" << ((r.out_soff - shift) / 8) << " + it] = acc;\n";
  if (track_max)
    o << "        lmax = max(lmax, max(__float_as_uint(acc.x) & 0x7fffffffu, __float_as_uint(acc.y) & 0x7fffffffu));\n";
  o << "      }\n";
  o << "    }\n";
}

}  // namespace

std::map<int, std::pair<int, int>> static_bounds(const ResidentLayout &L) {
  std::map<int, std::pair<int, int>> bound;  // metadata slot -> (k, exponent)
  std::map<int, int> depth;                  // chain depth
  for (const RStep &r : L.steps) {
    if (r.out_meta == L.final_meta) continue;
    int dp = 1, ex = 0;
    bool ok = true;
    for (int i = 0; i < r.m && ok; ++i) {
      if (r.in[i].meta < 0) continue;
      auto it = bound.find(r.in[i].meta);
      if (it == bound.end()) ok = false;
      else {
        dp = std::max(dp, depth[r.in[i].meta] + 1);
        ex += it->second.first + 1 + it->second.second;  // scale exponent k+1, recorded exponent
      }
    }
    if (ok && dp <= 3) {
      bound[r.out_meta] = {r.k, ex};
      depth[r.out_meta] = dp;
    }
  }
  return bound;
}

// CUDA source of the resident kernel specialised to layout L of plan p.
// mode RES_WHOLE: the whole pass per CTA.  RES_MAIN: the steps with a batch
// axis; the bitstring-independent tensors they read come from the pre
// region, written by the RES_PRE kernel (one CTA running the steps without a
// batch axis), which the main kernel may overlap up to the point where it
// waits for them (programmatic dependent launch).
std::string resident_source(const qgm_plan *p, const ResidentLayout &L, const std::string &name, int minb,
                            int mode) {
  std::ostringstream o;
  o << kPrelude;
  const int logBc = __builtin_ctz(L.chunk);
  const int64_t shift = worklist_bytes(L);
  const bool pre = mode == RES_PRE, main_part = mode == RES_MAIN;
  o << "extern \"C\" __global__ void __launch_bounds__(256, " << minb << ") " << name
    << "(const char *ws, const RJob *jobs, int n_jobs, const u64 *bits, long long B, double c_re, double c_im, "
       "double2 *out, Header *hdr) {\n";
  o << "  extern __shared__ __align__(16) char sm[];\n";
  o << "  float2 *F = reinterpret_cast<float2 *>(sm);\n";
  o << "  Meta *meta = reinterpret_cast<Meta *>(sm);\n";
  o << "  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;\n";
  o << "  const long long b0 = (long long)blockIdx.x * " << L.chunk << ";\n";
  if (pre) o << "  asm volatile(\"griddepcontrol.launch_dependents;\");\n";
  // shared memory starts as the plan's image: zeros (tensor metadata
  // included) with the bitstring-independent leaf rows in place
  const int64_t smem = compiled_smem(L);
  o << "  {\n    const uint4 *img = reinterpret_cast<const uint4 *>(ws + " << p->off_image << ");\n";
  o << "    uint4 *S = reinterpret_cast<uint4 *>(sm);\n";
  o << "#pragma unroll 4\n    for (int i = tid; i < " << smem / 16 << "; i += 256) S[i] = __ldg(img + i);\n  }\n";
  int n_batched = 0;
  for (const RJob &j : L.jobs) n_batched += j.batched != 0;
  if (!pre && n_batched) {
    // leaf rows that depend on the output bits of x_beta (listed first)
    o << "  __syncthreads();\n";
    o << "  const float2 *wsf = reinterpret_cast<const float2 *>(ws);\n";
    if (L.chunk == 1) o << "  const u64 x1 = b0 < B ? __ldg(bits + b0) : 0ull;\n";
    o << "  for (int t = tid; t < " << (n_batched << logBc) << "; t += 256) {\n";
    o << "    const int b = t & " << (L.chunk - 1) << ";\n";
    o << "    const RJob jb = jobs[t >> " << logBc << "];\n";
    o << "    int ob = 0;\n";
    o << "    if (jb.n_out) {\n";
    if (L.chunk == 1) o << "      const u64 x = x1;\n";
    else o << "      const u64 x = (b0 + b < B) ? bits[b0 + b] : 0ull;\n";
    o << "      ob = jb.n_out == 1 ? (int)((x >> jb.q0) & 1ull) : (int)((((x >> jb.q0) & 1ull) << 1) | ((x >> jb.q1) & 1ull));\n";
    o << "    }\n";
    o << "    reinterpret_cast<float2 *>(sm + jb.dst - " << shift << ")[b] = __ldg(wsf + jb.src + ob);\n";
    o << "  }\n";
  }
  if (main_part) {
    // the pre kernel's outputs and their scales, once it has finished
    o << "  __syncthreads();\n";
    o << "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n";
    o << "  {\n    const float2 *pd = reinterpret_cast<const float2 *>(ws + " << p->off_pre << ") + " << p->pre_data
      << ";\n";
    o << "    const int2 *pm = reinterpret_cast<const int2 *>(ws + " << p->off_pre << ");\n";
    for (size_t j = 0; j < L.pre.size(); ++j) {
      const auto &t = L.pre[j];
      o << "    for (int x = tid; x < " << t.entries << "; x += 256) F[" << ((t.soff - shift) / 8) << " + x] = pd["
        << t.goff << " + x];\n";
      o << "    if (tid == " << (j % 256) << ") { const int2 v = pm[" << j << "]; meta[" << t.meta
        << "].maxbits = (unsigned)v.x; meta[" << t.meta << "].exp = v.y; }\n";
    }
    o << "  }\n";
  }
  o << "  __syncthreads();\n";
  // recorded maxima known before the run: steps with a static bound
  const std::map<int, std::pair<int, int>> static_k = static_bounds(L);  // slot -> (k of 2^k, exponent)
  // steps in level order; inside a level grouped by first warp, so that
  // each warp's code for the level is contiguous
  std::vector<size_t> emit_order(L.steps.size());
  for (size_t q = 0; q < emit_order.size(); ++q) emit_order[q] = q;
  std::stable_sort(emit_order.begin(), emit_order.end(), [&](size_t a, size_t b) {
    if (L.level[a] != L.level[b]) return L.level[a] < L.level[b];
    return (L.steps[a].sched & 15) < (L.steps[b].sched & 15);
  });
  int cur_level = -1;
  for (size_t q : emit_order) {
    const RStep &r = L.steps[q];
    if ((pre && r.batched_out) || (main_part && !r.batched_out)) continue;
    if (L.level[q] != cur_level) {
      if (cur_level >= 0) o << "  __syncthreads();\n";
      cur_level = L.level[q];
    }
    const StepDesc &d = p->steps[L.src_step[q]];
    const int w0 = r.sched & 15, nw = (r.sched >> 4) & 15;
    o << "  // step " << L.src_step[q] << ": " << d.m << " inputs, " << d.k << " summed, " << d.w_out
      << " kept (level " << L.level[q] << ")\n";
    o << "  if (wid >= " << w0 << " && wid < " << (w0 + nw) << ") {\n";
    o << "    const int gt = tid - " << (32 * w0) << ";\n";
    // inputs whose producer has a static bound 2^k' get the constant scale
    // 2^-(k'+1) (exponent k'+1, recorded exponent 0); the others read theirs
    int es_static = 0, esum_static = 0;
    bool any_dynamic = false;
    for (int i = 0; i < d.m; ++i)
      if (r.in[i].meta >= 0) {
        auto it = static_k.find(r.in[i].meta);
        if (it != static_k.end()) {
          es_static += it->second.first + 1;
          esum_static += it->second.first + 1 + it->second.second;
        } else {
          any_dynamic = true;
        }
      }
    o << "    int es = " << es_static << ", esum = " << esum_static << ";\n";
    for (int i = 0; i < d.m; ++i) {
      if (r.in[i].meta < 0) continue;
      auto it = static_k.find(r.in[i].meta);
      if (it != static_k.end())
        o << "    const float s" << i << " = __int_as_float(" << (126 - it->second.first) << " << 23);\n";
      else
        o << "    float s" << i << "; { int e; opscale(meta, " << r.in[i].meta << ", s" << i
          << ", e, esum); es += e; }\n";
    }
    // scales: one combined factor per entry when the inputs' exponents sum
    // to a representable power of two; otherwise the intermediate inputs are
    // rescaled in place first (each feeds this step only) and the factor is 1
    bool any_meta = false;
    for (int i = 0; i < d.m; ++i) any_meta |= r.in[i].meta >= 0;
    o << "    float comb = 1.f;\n";
    if (any_meta && !any_dynamic && es_static >= -120 && es_static <= 120) {
      o << "    comb = __int_as_float(" << (127 - es_static) << " << 23);\n";
    } else if (any_meta) {
      o << "    if (es >= -120 && es <= 120) comb = __int_as_float((127 - es) << 23);\n";
      o << "    else {\n";
      for (int i = 0; i < d.m; ++i) {
        if (r.in[i].meta < 0) continue;
        const SymTensor &t = p->sim.tensors[p->sim.steps[L.src_step[q]].inputs[i]];
        const int64_t n = ((int64_t)1 << t.vars.size()) * (t.batched ? L.chunk : 1);
        o << "      for (int x = gt; x < " << n << "; x += " << 32 * nw << ") { float2 &y = F["
          << ((r.in[i].soff - shift) / 8) << " + x]; y.x *= s" << i << "; y.y *= s" << i << "; }\n";
      }
      if (nw > 1) o << "      asm volatile(\"bar.sync %0, %1;\" :: \"r\"(" << (1 + w0) << "), \"r\"(" << 32 * nw << "));\n";
      else o << "      __syncwarp();\n";
      o << "    }\n";
    }
    const bool track = static_k.count(r.out_meta) == 0;
    {
      std::ostringstream b;
      emit_body(b, p, L, q, shift, track);
      if (track) o << "    unsigned lm;\n    {\n" << b.str() << "    lm = lmax; }\n";
      else o << "    {\n" << b.str() << "    }\n";
    }
    if (track) {
      // max |re|,|im| over the step's entries: non-negative floats (and NaN,
      // which must reach the maximum) order like their bit patterns
      o << "    lm = __reduce_max_sync(0xffffffffu, lm);\n";
      o << "    if (lane == 0) {\n";
      o << "      if (lm) atomicMax(&meta[" << r.out_meta << "].maxbits, lm);\n";
      o << "      if (wid == " << w0 << ") meta[" << r.out_meta << "].exp = esum;\n";
      o << "    }\n";
    }
    o << "  }\n";
  }
  o << "  __syncthreads();\n";
  if (pre) {
    // publish the outputs read by batched steps, with their scales
    o << "  {\n    float2 *pd = reinterpret_cast<float2 *>(const_cast<char *>(ws) + " << p->off_pre << ") + "
      << p->pre_data << ";\n";
    o << "    int2 *pm = reinterpret_cast<int2 *>(const_cast<char *>(ws) + " << p->off_pre << ");\n";
    for (size_t j = 0; j < L.pre.size(); ++j) {
      const auto &t = L.pre[j];
      o << "    for (int x = tid; x < " << t.entries << "; x += 256) pd[" << t.goff << " + x] = F["
        << ((t.soff - shift) / 8) << " + x];\n";
      o << "    if (tid == " << (j % 256) << ") pm[" << j << "] = make_int2((int)meta[" << t.meta << "].maxbits, meta["
        << t.meta << "].exp);\n";
    }
    o << "  }\n}\n";
    return o.str();
  }
  o << "  if (tid == 0 && ((meta[" << L.final_meta << "].maxbits >> 23) & 0xff) == 0xff) atomicCAS(&hdr->status, 0, -5);\n";
  o << "  if (tid < " << L.chunk << " && b0 + tid < B) {\n";
  o << "    const float2 v = F[" << ((L.final_soff - shift) / 8) << (p->final_batched ? " + tid" : "") << "];\n";
  o << "    const double scl = ldexp(1.0, meta[" << L.final_meta << "].exp);\n";
  o << "    const double re = (double)v.x * scl, im = (double)v.y * scl;\n";
  o << "    out[b0 + tid] = make_double2(re * c_re - im * c_im, re * c_im + im * c_re);\n";
  o << "  }\n}\n";
  return o.str();
}

}  // namespace qgm

// ---------------------------------------------------------------- NVRTC
namespace qgm {

namespace {

struct Nvrtc {
  bool ok = false;
  int (*create)(void **, const char *, const char *, int, const char *const *, const char *const *) = nullptr;
  int (*compile)(void *, int, const char *const *) = nullptr;
  int (*log_size)(void *, size_t *) = nullptr;
  int (*log)(void *, char *) = nullptr;
  int (*cubin_size)(void *, size_t *) = nullptr;
  int (*cubin)(void *, char *) = nullptr;
  int (*destroy)(void **) = nullptr;
};

Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    void *h = nullptr;
    for (const char *name : {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"})
      if ((h = dlopen(name, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) return;
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
  });
  return n;
}

struct CacheKey {
  int device;
  size_t hash, len;
  bool operator<(const CacheKey &o) const {
    return device != o.device ? device < o.device : hash != o.hash ? hash < o.hash : len < o.len;
  }
};

std::mutex g_cache_mu;
std::map<CacheKey, cudaKernel_t> g_cache;

}  // namespace

// Compile `src` for the current device (sm_103a) and return kernel `name`.
// Kernels are cached per device and source for the life of the process.
// Returns false (with a message in *err) when NVRTC is unavailable or the
// compile or load fails.
bool jit_kernel(const std::string &src, const std::string &name, int device, cudaKernel_t *out,
                std::string *err) {
  const CacheKey key{device, std::hash<std::string>()(src), src.size()};
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      return true;
    }
  }
  Nvrtc &n = nvrtc();
  if (!n.ok) {
    *err = "NVRTC library not found";
    return false;
  }
  void *prog = nullptr;
  if (n.create(&prog, src.c_str(), "qgm_resident.cu", 0, nullptr, nullptr) != 0) {
    *err = "nvrtcCreateProgram failed";
    return false;
  }
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
  const int rc = n.compile(prog, 3, opts);
  if (rc != 0) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    *err = "NVRTC compile failed: " + log.substr(0, 2000);
    n.destroy(&prog);
    return false;
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  std::vector<char> cubin(cs);
  n.cubin(prog, cubin.data());
  n.destroy(&prog);
  cudaLibrary_t lib;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) {
    *err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
    return false;
  }
  cudaKernel_t k;
  e = cudaLibraryGetKernel(&k, lib, name.c_str());
  if (e != cudaSuccess) {
    *err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
    return false;
  }
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache[key] = k;
  *out = k;
  return true;
}

}  // namespace qgm
