// C ABI of the mfIPM library (declarations and contracts in include/mfipm.h):
// argument validation, workspace layout, cluster-size choice and launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <string>
#include <vector>

#include "dct_gen.h"
#include "device_common.cuh"
#include "internal.h"
#include "large_dct.h"
#include "mrhs.h"

namespace mfipm {
// Kernels launched by the current public call on this thread (kept in mrhs.cu, where the
// lockstep solvers count theirs): cleared when a solve, batched solve or backward call
// starts; the persistent path adds its launches.
void lockstep_stats_reset();
void note_launches(int64_t n);
}  // namespace mfipm

using namespace mfipm;

namespace {

thread_local std::string g_err;

// Plain CUDA-core GEMM instead of tcgen05 in the bf16 solver (mfipm_set_gemm_mode; for tests).
bool g_force_simple_gemm = false;
// Residual of the bf16 solver: exact digit slices on the tensor cores (1) or the biased float32
// accumulator on the CUDA cores (0) (mfipm_set_residual_mode).
int g_resid_tc = 1;

// Autotuner results (mfipm_autotune), process-wide.  Persistent partial-DCT kernel: keyed by
// the batch's largest n and ceil(log2 batch) -> cluster size G and the largest n solved by a
// single CTA.  Shared bf16 A: keyed by (m, n, right-hand sides) -> split-K of the two GEMMs.
struct TuneDct {
  int G;
  int64_t cta_max_n;
};
struct TuneGemm {
  int s1, s2, st1, st2;  // split-K and ring stages of T = A W and Y = A^T T
};
std::mutex g_tune_mu;
std::map<std::pair<int64_t, int>, TuneDct> g_tune_dct;
std::map<std::tuple<int64_t, int64_t, int>, TuneGemm> g_tune_gemm;
int ceil_log2i(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v) ++l;
  return l;
}

// Side stream and fork/join events of the single-CTA helper launch (created on first use).
thread_local cudaStream_t g_side = nullptr;
thread_local cudaEvent_t g_fork = nullptr, g_join = nullptr;

// Optional timing of the solver kernel (mfipm_set_timing / mfipm_last_kernel_ms).
thread_local bool g_timing = false;
thread_local cudaEvent_t g_ev[2] = {nullptr, nullptr};
thread_local float g_last_ms = -1.0f;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(MFIPM_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ilog2(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v) ++l;
  return l;
}
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

constexpr int64_t kDctMinN = 64, kDctMaxN = 65536;
constexpr int64_t kDenseMaxM = 6144;

// Partial-DCT problems with n >= this go to the lockstep multi-pass solver (large_dct.cu);
// the rest to the cluster-resident persistent kernel (mfipm_set_large_dct_threshold).
int64_t g_large_dct_min_n = 2 * kDctMaxN;
bool is_large_dct(const mfipm_operator& o) {
  return o.kind == MFIPM_OP_PARTIAL_DCT && is_pow2(o.n) && o.n >= g_large_dct_min_n && o.n >= kLdMinN;
}

// Partial DCT of a general length (the mixed-radix chain, one CTA per problem): n even in
// [8, 16384] with n/2 free of prime factors above 5.
constexpr int64_t kGenMinN = 8, kGenMaxN = 16384;
bool is_gen_dct_n(int64_t n) {
  if (n < kGenMinN || n > kGenMaxN || (n & 1)) return false;
  int64_t r = n / 2;
  for (int f : {2, 3, 5})
    while (r % f == 0) r /= f;
  return r == 1;
}
// a partial-DCT batch with a length that is not a power of two runs on the mixed-radix chain
bool needs_gen(const mfipm_operator* ops, int batch) {
  for (int i = 0; i < batch; ++i)
    if (ops[i].kind == MFIPM_OP_PARTIAL_DCT && !is_pow2(ops[i].n)) return true;
  return false;
}

int validate_op(const mfipm_operator* op, int idx) {
  if (!op) return fail(MFIPM_INVALID_ARG, "operator %d is NULL", idx);
  if (op->m < 0 || op->n <= 0 || op->m > op->n)
    return fail(MFIPM_INVALID_ARG, "operator %d: need 0 <= m <= n, n > 0 (m=%lld n=%lld)", idx,
                (long long)op->m, (long long)op->n);
  if (op->kind == MFIPM_OP_PARTIAL_DCT) {
    const bool pow2 = is_pow2(op->n) && op->n >= kDctMinN && op->n <= kLdMaxN;
    if (!pow2 && !is_gen_dct_n(op->n))
      return fail(MFIPM_INVALID_ARG,
                  "operator %d: partial DCT needs n a power of two in [%lld, %lld], or an even n in [%lld, %lld] "
                  "whose half has no prime factor above 5 (n=%lld)",
                  idx, (long long)kDctMinN, (long long)kLdMaxN, (long long)kGenMinN, (long long)kGenMaxN,
                  (long long)op->n);
    if (op->m > 0 && !op->rows) return fail(MFIPM_INVALID_ARG, "operator %d: rows is NULL", idx);
    return MFIPM_OK;
  }
  if (op->kind == MFIPM_OP_PARTIAL_HAAR) {
    if (!is_pow2(op->n) || op->n < kDctMinN || op->n > kDctMaxN)
      return fail(MFIPM_INVALID_ARG, "operator %d: partial Haar needs n a power of two in [%lld, %lld] (n=%lld)",
                  idx, (long long)kDctMinN, (long long)kDctMaxN, (long long)op->n);
    if (op->m > 0 && !op->rows) return fail(MFIPM_INVALID_ARG, "operator %d: rows is NULL", idx);
    return MFIPM_OK;
  }
  if (op->kind == MFIPM_OP_DENSE) {
    if (op->m > 0 && !op->A) return fail(MFIPM_INVALID_ARG, "operator %d: A is NULL", idx);
    if (op->lda < op->n) return fail(MFIPM_INVALID_ARG, "operator %d: lda < n", idx);
    if (!(op->a_scale > 0.0) || !isfinite(op->a_scale))
      return fail(MFIPM_INVALID_ARG, "operator %d: a_scale must be positive and finite", idx);
    if (op->a_dtype == MFIPM_A_BF16) return MFIPM_OK;  // shared-A multi-RHS solver
    if (op->a_dtype != MFIPM_A_F64)
      return fail(MFIPM_UNSUPPORTED, "operator %d: dense A must be float64 or bf16 (a_dtype=%d)", idx, op->a_dtype);
    if (op->m > kDenseMaxM)
      return fail(MFIPM_UNSUPPORTED, "operator %d: dense m=%lld above %lld for the per-problem solver", idx,
                  (long long)op->m, (long long)kDenseMaxM);
    return MFIPM_OK;
  }
  return fail(MFIPM_INVALID_ARG, "operator %d: unknown kind %d", idx, op->kind);
}

int validate_params(const mfipm_params* p) {
  if (!p) return fail(MFIPM_INVALID_ARG, "params is NULL");
  if (!(p->tol > 0) || !(p->tol_pcg > 0) || p->max_iter < 1 || p->max_iter_pcg < 1)
    return fail(MFIPM_INVALID_ARG, "params: tol, tol_pcg must be > 0 and iteration caps >= 1");
  if (!(p->eta > 0 && p->eta < 1)) return fail(MFIPM_INVALID_ARG, "params: eta must be in (0,1)");
  if (!(p->sigma1 >= 0 && p->sigma2 >= 0 && p->sigma3 >= 0 && p->sigma1 <= 1 && p->sigma2 <= 1 && p->sigma3 <= 1))
    return fail(MFIPM_INVALID_ARG, "params: sigma values must lie in [0,1]");
  if (p->precision < 0 || p->precision > 2) return fail(MFIPM_INVALID_ARG, "params: bad precision %d", p->precision);
  if (p->outer != MFIPM_OUTER_DF && p->outer != MFIPM_OUTER_FP64)
    return fail(MFIPM_INVALID_ARG, "params: bad outer-loop arithmetic %d", p->outer);
  if (!(p->outer_f32_gap >= 0) || !isfinite(p->outer_f32_gap))
    return fail(MFIPM_INVALID_ARG, "params: outer_f32_gap must be finite and >= 0");
  if (p->centrality_correctors < 0 || p->centrality_correctors > 16)
    return fail(MFIPM_INVALID_ARG, "params: centrality_correctors must lie in [0, 16]");
  const int cs = p->cluster_size;
  if (!(cs == 0 || cs == 1 || cs == 2 || cs == 4 || cs == 8 || cs == 16))
    return fail(MFIPM_INVALID_ARG, "params: cluster_size must be 0,1,2,4,8,16");
  return MFIPM_OK;
}

SolveParams to_solve(const mfipm_params* p) {
  SolveParams s{};
  s.tol = p->tol;
  s.tol_pcg = p->tol_pcg;
  s.sigma1 = p->sigma1;
  s.sigma2 = p->sigma2;
  s.sigma3 = p->sigma3;
  s.alpha_bar = p->alpha_bar;
  s.alpha_tilde = p->alpha_tilde;
  s.eta = p->eta;
  s.max_iter = p->max_iter;
  s.max_iter_pcg = p->max_iter_pcg;
  s.equal_steps = p->equal_steps;
  s.resid_fp64 = p->outer == MFIPM_OUTER_FP64;
  s.f32_gap = p->outer_f32_gap;
  s.mcc = p->centrality_correctors;
  s.mcc_beta_min = 0.1;
  s.mcc_beta_max = 10.0;
  s.mcc_delta = 0.1;
  s.mcc_gamma = 0.1;
  return s;
}

// Largest cluster size that the DCT chain supports for length n: shared memory holds
// 12 n / G bytes (<= 192 KiB) and every CTA needs >= 1 exchange slot (n >= 4 G^2).
int dct_min_G(int64_t n) { return (int)std::max<int64_t>(1, n / 16384); }
int dct_max_G(int64_t n) {
  int g = 16;
  while (g > 1 && n < 4 * (int64_t)g * g) g >>= 1;
  return g;
}

// Per-problem bytes of the device state (excluding shared tables).
size_t problem_bytes(const mfipm_operator& op, bool pcg64) {
  const size_t n = (size_t)op.n;
  size_t b = 0;
  if (op.kind == MFIPM_OP_PARTIAL_DCT || op.kind == MFIPM_OP_PARTIAL_HAAR)
    b += align256(n) + 2 * align256(8 * n);  // mask, bsu, bsu_df
  if (op.kind == MFIPM_OP_PARTIAL_DCT) b += align256(n / 2) + align256(16 * n);  // mcode, bpk
  b += align256(32 * n);                                                     // z, s
  b += align256(6 * n * (pcg64 ? 16 : 8));                                   // x1 x2 r p d xc
  b += align256(8 * n);                                                      // scratch (apply)
  return b;
}

struct Layout {
  size_t off_hdr, off_tw64, off_tw32, off_twdf, off_desc, off_info, off_gtau, off_twg, off_probs, total;
  int log2_tw;
  std::vector<std::pair<int64_t, size_t>> gen_tabs;  // mixed-radix chain: (n, offset of its roots table)
};

Layout make_layout(const mfipm_operator* ops, int batch, bool pcg64) {
  Layout L{};
  int64_t max_dct = 0;
  for (int i = 0; i < batch; ++i)
    if (ops[i].kind == MFIPM_OP_PARTIAL_DCT) max_dct = std::max<int64_t>(max_dct, ops[i].n);
  L.log2_tw = max_dct ? ilog2(max_dct) + 2 : 6;
  size_t o = 0;
  L.off_hdr = o;
  o += 256;
  L.off_tw64 = o;  // level-ordered tables: 2^(log2_tw+1) entries each
  o += align256(((size_t)2 << L.log2_tw) * 16);
  L.off_tw32 = o;
  o += align256(((size_t)2 << L.log2_tw) * 8);
  L.off_twdf = o;
  o += align256(((size_t)2 << L.log2_tw) * 16);
  L.off_desc = o;
  o += align256(sizeof(ProbDesc) * (size_t)batch);
  L.off_info = o;
  o += align256(sizeof(mfipm_info) * (size_t)batch);
  L.off_gtau = o;
  o += align256(sizeof(double) * (size_t)batch);
  L.off_twg = o;
  if (needs_gen(ops, batch))
    for (int i = 0; i < batch; ++i) {
      const int64_t n = ops[i].n;
      if (ops[i].kind != MFIPM_OP_PARTIAL_DCT || n > kGenMaxN) continue;
      bool seen = false;
      for (auto& t : L.gen_tabs) seen |= t.first == n;
      if (seen) continue;
      L.gen_tabs.push_back({n, o});
      o += align256(gen_tw_bytes(n / 2));
    }
  L.off_probs = o;
  for (int i = 0; i < batch; ++i) o += problem_bytes(ops[i], pcg64);
  L.total = o;
  return L;
}

bool pcg_in_fp64(const mfipm_operator& op, const mfipm_params* p) {
  (void)op;  // dense, partial DCT and partial Haar alike
  return p->precision == MFIPM_PREC_FP64;
}

int pick_G(const std::vector<mfipm_operator>& ops, const mfipm_params* p, int batch) {
  // the Haar chain follows the DCT's rule: the same shared memory per value and cluster sizes
  const bool dct = ops[0].kind == MFIPM_OP_PARTIAL_DCT || ops[0].kind == MFIPM_OP_PARTIAL_HAAR;
  int64_t max_n = 0, min_n = INT64_MAX;
  for (auto& o : ops) {
    max_n = std::max<int64_t>(max_n, o.n);
    min_n = std::min<int64_t>(min_n, o.n);
  }
  if (p->cluster_size) return p->cluster_size;
  if (dct) {
    int g;
    if (batch == 1) {
      g = (int)std::min<int64_t>(16, std::max<int64_t>(1, max_n / 2048));
    } else {
      g = dct_min_G(max_n);
    }
    g = std::max(g, dct_min_G(max_n));
    g = std::min(g, dct_max_G(min_n));
    return g;
  }
  // dense: columns per CTA >= 32
  int g = 16;
  while (g > 1 && min_n < 32 * (int64_t)g) g >>= 1;
  if (batch > 1) g = std::min(g, 4);
  return g;
}

// The bf16 shared-A multi-RHS path: every operator dense bf16 with the same A, m, n, lda = n
// and a_scale, and precision MFIPM_PREC_BF16_A.
int check_shared_bf16(const mfipm_operator* ops, int batch, const mfipm_params* p, bool* is_shared) {
  *is_shared = false;
  bool any_bf16 = false;
  for (int i = 0; i < batch; ++i) any_bf16 |= ops[i].kind == MFIPM_OP_DENSE && ops[i].a_dtype == MFIPM_A_BF16;
  if (!any_bf16 && p->precision != MFIPM_PREC_BF16_A) return MFIPM_OK;
  if (p->precision != MFIPM_PREC_BF16_A)
    return fail(MFIPM_UNSUPPORTED, "bf16 A needs precision MFIPM_PREC_BF16_A (the shared-A multi-RHS solver)");
  for (int i = 0; i < batch; ++i) {
    const mfipm_operator& o = ops[i];
    if (o.kind != MFIPM_OP_DENSE || o.a_dtype != MFIPM_A_BF16)
      return fail(MFIPM_UNSUPPORTED, "MFIPM_PREC_BF16_A needs dense bf16 operators (operator %d)", i);
    if (o.A != ops[0].A || o.m != ops[0].m || o.n != ops[0].n || o.a_scale != ops[0].a_scale || o.lda != ops[0].lda)
      return fail(MFIPM_UNSUPPORTED, "the bf16 solver shares one A between right-hand sides (operator %d differs)", i);
    if (o.lda != o.n) return fail(MFIPM_UNSUPPORTED, "bf16 A must be packed (lda == n)");
    if (o.m < 1) return fail(MFIPM_INVALID_ARG, "bf16 A needs m >= 1");
  }
  *is_shared = true;
  return MFIPM_OK;
}

struct Prepared {
  Layout lay;
  std::vector<ProbDesc> desc;
  KernelArgs args;
  int G;
  bool dct, haar, pcg64;  // dct: a masked orthonormal operator (partial DCT or partial Haar)
  bool gen;               // partial DCT on the mixed-radix chain (a length not a power of two)
  int64_t max_n, max_m;
  int64_t cta_max_n = 0;  // > 0: largest n solved by a single CTA (tuned), else the default rule
  char* ws;
};

int prepare(int batch, const mfipm_operator* ops, const double* const* b, const double* tau,
            const mfipm_params* p, double* const* x, double* const* zs_out, void* workspace, size_t ws_bytes,
            Prepared& P) {
  if (batch < 1) return fail(MFIPM_INVALID_ARG, "batch must be >= 1");
  if (!ops || !b || !tau || !x) return fail(MFIPM_INVALID_ARG, "NULL argument array");
  int rc = validate_params(p);
  if (rc) return rc;
  std::vector<mfipm_operator> vops(ops, ops + batch);
  const int kind = ops[0].kind;
  for (int i = 0; i < batch; ++i) {
    if ((rc = validate_op(&ops[i], i))) return rc;
    if (ops[i].kind != kind) return fail(MFIPM_UNSUPPORTED, "a batch must use one operator kind");
    if (!(tau[i] > 0.0) || !isfinite(tau[i])) return fail(MFIPM_INVALID_ARG, "tau[%d] must be positive and finite", i);
    if (ops[i].m > 0 && !b[i]) return fail(MFIPM_INVALID_ARG, "b[%d] is NULL", i);
    if (!x[i]) return fail(MFIPM_INVALID_ARG, "x[%d] is NULL", i);
  }
  for (int i = 0; i < batch; ++i)
    if (ops[i].kind == MFIPM_OP_DENSE && ops[i].a_dtype == MFIPM_A_BF16)
      return fail(MFIPM_UNSUPPORTED, "bf16 A is solved by the shared-A multi-RHS solver (precision MFIPM_PREC_BF16_A)");
  P.haar = kind == MFIPM_OP_PARTIAL_HAAR;
  P.dct = kind == MFIPM_OP_PARTIAL_DCT || P.haar;
  P.gen = kind == MFIPM_OP_PARTIAL_DCT && needs_gen(ops, batch);
  if (P.gen) {
    for (int i = 0; i < batch; ++i)
      if (ops[i].n > kGenMaxN)
        return fail(MFIPM_UNSUPPORTED, "operator %d: a batch with a partial DCT whose n is not a power of two runs one "
                    "CTA per problem, n <= %lld (n=%lld)", i, (long long)kGenMaxN, (long long)ops[i].n);
    if (p->cluster_size > 1)
      return fail(MFIPM_INVALID_ARG, "cluster_size %d: the partial DCT of a general length runs one CTA per problem",
                  p->cluster_size);
  }
  for (int i = 0; i < batch; ++i)
    if (P.dct && ops[i].n > kDctMaxN)
      return fail(MFIPM_UNSUPPORTED, "operator %d: n=%lld above the cluster solver's %lld", i, (long long)ops[i].n,
                  (long long)kDctMaxN);
  if (P.dct && p->precision != MFIPM_PREC_FP32_PCG && p->precision != MFIPM_PREC_FP64)
    return fail(MFIPM_UNSUPPORTED, "the partial-DCT and partial-Haar solvers run their PCG in float32 or float64 "
                "(precision=%d)", p->precision);
  if (P.haar && p->outer != MFIPM_OUTER_DF)
    return fail(MFIPM_UNSUPPORTED, "the partial-Haar solver keeps its iterate in double-float (outer=%d)", p->outer);
  if (!P.dct && p->precision == MFIPM_PREC_BF16_A)
    return fail(MFIPM_UNSUPPORTED, "bf16 dense A goes through the shared-A multi-RHS solver");
  P.pcg64 = pcg_in_fp64(ops[0], p);
  P.lay = make_layout(ops, batch, P.pcg64);
  if (!workspace) return fail(MFIPM_INVALID_ARG, "workspace is NULL");
  if (((uintptr_t)workspace & 255) != 0) return fail(MFIPM_INVALID_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < P.lay.total)
    return fail(MFIPM_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, P.lay.total);
  P.max_n = 0;
  P.max_m = 0;
  for (auto& o : vops) {
    P.max_n = std::max<int64_t>(P.max_n, o.n);
    P.max_m = std::max<int64_t>(P.max_m, o.m);
  }
  P.G = P.gen ? 1 : pick_G(vops, p, batch);
  if (P.dct && !P.haar && !P.gen && p->cluster_size == 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_dct.find({P.max_n, ceil_log2i(batch)});
    if (it != g_tune_dct.end()) {
      int64_t min_n = INT64_MAX;
      for (auto& o : vops) min_n = std::min<int64_t>(min_n, o.n);
      if (it->second.G >= dct_min_G(P.max_n) && it->second.G <= dct_max_G(min_n)) {
        P.G = it->second.G;
        P.cta_max_n = it->second.cta_max_n;
      }
    }
  }
  if (P.dct) {
    int64_t min_n = INT64_MAX;
    for (auto& o : vops) min_n = std::min<int64_t>(min_n, o.n);
    if (P.G < dct_min_G(P.max_n) || P.G > dct_max_G(min_n))
      return fail(MFIPM_INVALID_ARG, "cluster_size %d does not fit n in [%lld, %lld]", P.G, (long long)min_n,
                  (long long)P.max_n);
  } else if ((P.max_n + P.G - 1) / P.G > 16384) {
    return fail(MFIPM_UNSUPPORTED, "dense n=%lld too large for cluster size %d", (long long)P.max_n, P.G);
  }
  char* ws = static_cast<char*>(workspace);
  P.ws = ws;
  P.desc.resize(batch);
  size_t o = P.lay.off_probs;
  mfipm_info* info_dev = reinterpret_cast<mfipm_info*>(ws + P.lay.off_info);
  for (int i = 0; i < batch; ++i) {
    ProbDesc& d = P.desc[i];
    memset(&d, 0, sizeof(d));
    const mfipm_operator& op = ops[i];
    const size_t n = (size_t)op.n;
    d.n = op.n;
    d.m = op.m;
    d.kind = op.kind;
    d.log2n = ilog2(op.n);
    d.tau = tau[i];
    d.b = b[i];
    d.x_out = x[i];
    d.zs_out = zs_out ? zs_out[i] : nullptr;
    d.rows = op.rows;
    d.A = op.A;
    d.a_dtype = op.a_dtype;
    d.a_scale = op.a_scale;
    d.lda = op.lda;
    size_t q = o;
    if (P.dct) {
      d.mask = reinterpret_cast<uint8_t*>(ws + q);
      q += align256(n);
      d.bsu = reinterpret_cast<double*>(ws + q);
      q += align256(8 * n);
      d.bsu_df = reinterpret_cast<float2*>(ws + q);
      q += align256(8 * n);
      if (!P.haar) {
        d.mcode = reinterpret_cast<uint8_t*>(ws + q);
        q += align256(n / 2);
        d.bpk = ws + q;
        q += align256(16 * n);
      }
      if (P.gen)
        for (auto& t : P.lay.gen_tabs)
          if (t.first == op.n) d.twg = ws + t.second;
    }
    d.zs = reinterpret_cast<double*>(ws + q);
    q += align256(32 * n);
    d.pcg = ws + q;
    q += align256(6 * n * (P.pcg64 ? 16 : 8));
    d.scratch = reinterpret_cast<double*>(ws + q);
    q += align256(8 * n);
    d.grad_tau = reinterpret_cast<double*>(ws + P.lay.off_gtau) + i;
    d.info = info_dev + i;
    o += problem_bytes(op, P.pcg64);
  }
  KernelArgs& a = P.args;
  memset(&a, 0, sizeof(a));
  a.probs = reinterpret_cast<const ProbDesc*>(ws + P.lay.off_desc);
  a.batch = batch;
  a.queue = reinterpret_cast<int*>(ws + P.lay.off_hdr);
  a.err = reinterpret_cast<int*>(ws + P.lay.off_hdr + 64);  // queue counters occupy bytes 0..7
  a.tw64 = reinterpret_cast<const double2*>(ws + P.lay.off_tw64);
  a.tw32 = reinterpret_cast<const float2*>(ws + P.lay.off_tw32);
  a.twdf = reinterpret_cast<const float4*>(ws + P.lay.off_twdf);
  a.log2_tw = P.lay.log2_tw;
  a.prm = to_solve(p);
  if (P.dct && !P.haar && P.pcg64) a.prm.resid_fp64 = 1;  // the DCT's float64 PCG runs with the float64 outer loop
  return MFIPM_OK;
}

int run(Prepared& P, cudaStream_t st, int batch, mfipm_info* infos, const std::vector<int>* order,
        bool allow_timing = true) {
  const bool timing = g_timing && allow_timing;
  cudaError_t e;
  // work queue in cost order (largest first): the descriptor array is permuted, infos are not
  std::vector<ProbDesc> sorted(P.desc);
  if (order) {
    for (int i = 0; i < batch; ++i) sorted[i] = P.desc[(*order)[i]];
  }
  if ((e = cudaMemcpyAsync(P.ws + P.lay.off_desc, sorted.data(), sizeof(ProbDesc) * batch, cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cuda_fail(e, "upload descriptors");
  if ((e = cudaMemsetAsync(P.ws + P.lay.off_hdr, 0, 256, st)) != cudaSuccess) return cuda_fail(e, "clear header");
  if (P.dct) {
    if ((e = launch_twiddles(const_cast<double2*>(P.args.tw64), const_cast<float2*>(P.args.tw32),
                             const_cast<float4*>(P.args.twdf), P.args.log2_tw, st)) != cudaSuccess)
      return cuda_fail(e, "twiddle kernel");
    if ((e = launch_dct_setup(P.args.probs, batch, P.max_n, P.args.err, st, P.args.prm.resid_fp64 != 0)) !=
        cudaSuccess)
      return cuda_fail(e, "setup kernel");
  }
  if (P.gen)
    for (auto& t : P.lay.gen_tabs)
      if ((e = launch_gen_twiddles(P.ws + t.second, t.first, st)) != cudaSuccess) return cuda_fail(e, "roots table");
  // problems small enough for one CTA's shared memory go to the per-CTA phase of the kernel
  // (the queue order puts every cluster problem before them)
  int nbig = batch;
  if (P.G == 1) {
    nbig = 0;
  } else if (P.dct) {
    int64_t small_max = std::min<int64_t>(16384, P.max_n / P.G);  // shared memory of one CTA
    if (P.cta_max_n > 0) small_max = std::min<int64_t>(small_max, P.cta_max_n);
    nbig = 0;
    for (int i = 0; i < batch; ++i) nbig += sorted[i].n > small_max;
  }
  P.args.nbig = nbig;
  const bool f64 = P.args.prm.resid_fp64 != 0;
  const int gen_variant = P.pcg64 ? kGenF64Pcg : f64 ? kGenF64 : kGenDF;
  int maxc = P.gen              ? max_active_ctas_dct_gen(gen_variant, P.max_n)
             : P.haar           ? (P.pcg64 ? max_active_clusters_haar_f64pcg(P.G, P.max_n)
                                           : max_active_clusters_haar(P.G, P.max_n))
             : P.dct && P.pcg64 ? max_active_clusters_dct_f64pcg(P.G, P.max_n)
             : P.dct ? (f64 ? max_active_clusters_dct_f64(P.G, P.max_n) : max_active_clusters_dct_df(P.G, P.max_n))
                     : max_active_clusters_dense(P.G, P.pcg64, P.max_n, P.max_m);
  if (maxc < 1) return fail(MFIPM_UNSUPPORTED, "no resident cluster of size %d fits this problem", P.G);
  const int clusters = std::min(maxc, std::max(nbig, (batch + P.G - 1) / P.G));
  if (timing) {
    for (auto& ev : g_ev)
      if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "timing event");
    cudaEventRecord(g_ev[0], st);
  }
  // SMs that no cluster of the persistent launch can hold (cluster placement leaves some of
  // them out) serve the per-CTA queue through a helper launch of single CTAs on a side stream
  int helper = 0;
  int64_t small_n = 0;
  if (P.dct && P.G > 1 && nbig < batch) {
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "device attributes");
    helper = std::min(sms - clusters * P.G, batch - nbig);
    for (int i = nbig; i < batch; ++i) small_n = std::max<int64_t>(small_n, sorted[i].n);
    if (helper > 0) {
      if (!g_side && (e = cudaStreamCreateWithFlags(&g_side, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "side stream");
      if ((!g_fork && (e = cudaEventCreateWithFlags(&g_fork, cudaEventDisableTiming)) != cudaSuccess) ||
          (!g_join && (e = cudaEventCreateWithFlags(&g_join, cudaEventDisableTiming)) != cudaSuccess))
        return cuda_fail(e, "helper events");
      if ((e = cudaEventRecord(g_fork, st)) != cudaSuccess) return cuda_fail(e, "fork");
    }
  }
  e = P.gen              ? launch_dct_gen_solver(gen_variant, P.args, P.max_n, clusters, st)
      : P.haar           ? (P.pcg64 ? launch_haar_solver_f64pcg(P.G, P.args, P.max_n, clusters, st)
                                    : launch_haar_solver(P.G, P.args, P.max_n, clusters, st))
      : P.dct && P.pcg64 ? launch_dct_solver_f64pcg(P.G, P.args, P.max_n, clusters, st)
      : P.dct ? (f64 ? launch_dct_solver_f64(P.G, P.args, P.max_n, clusters, st)
                     : launch_dct_solver_df(P.G, P.args, P.max_n, clusters, st))
              : launch_dense_solver(P.G, P.pcg64, P.args, P.max_n, P.max_m, clusters, st);
  if (e != cudaSuccess) return cuda_fail(e, "solver launch");
  if (helper > 0) {
    KernelArgs ha = P.args;
    ha.phase2_only = 1;
    if ((e = cudaStreamWaitEvent(g_side, g_fork, 0)) != cudaSuccess) return cuda_fail(e, "fork");
    e = P.haar             ? (P.pcg64 ? launch_haar_solver_f64pcg(1, ha, small_n, helper, g_side)
                                      : launch_haar_solver(1, ha, small_n, helper, g_side))
        : P.pcg64 ? launch_dct_solver_f64pcg(1, ha, small_n, helper, g_side)
        : f64     ? launch_dct_solver_f64(1, ha, small_n, helper, g_side)
                  : launch_dct_solver_df(1, ha, small_n, helper, g_side);
    if (e != cudaSuccess) return cuda_fail(e, "helper launch");
    if ((e = cudaEventRecord(g_join, g_side)) != cudaSuccess || (e = cudaStreamWaitEvent(st, g_join, 0)) != cudaSuccess)
      return cuda_fail(e, "join");
  }
  if (timing) cudaEventRecord(g_ev[1], st);
  // twiddles, mask/b setup, scatter, per-frequency packing, the roots tables of general
  // lengths, the solver and its helper launch
  note_launches((P.dct ? 4 + (int64_t)P.lay.gen_tabs.size() : 0) + 1 + (helper > 0 ? 1 : 0));
  int err = 0;
  if ((e = cudaMemcpyAsync(&err, P.args.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "read error word");
  if (infos) {
    if ((e = cudaMemcpyAsync(infos, P.ws + P.lay.off_info, sizeof(mfipm_info) * batch, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return cuda_fail(e, "read infos");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "solve");
  if (timing) {
    float ms = -1.0f;
    if (cudaEventElapsedTime(&ms, g_ev[0], g_ev[1]) == cudaSuccess) g_last_ms = ms;
  }
  if (err == -1) return fail(MFIPM_INVALID_ARG, "rows must be distinct, ascending and inside [0, n)");
  if (err == -2) return fail(MFIPM_NUMERIC, "b contains a non-finite value");
  if (err > 0 && infos) {
    for (int i = 0; i < batch; ++i)
      if (infos[i].status != MFIPM_OK) return infos[i].status;
  }
  return err > 0 ? err : MFIPM_OK;
}

std::vector<int> cost_order(const mfipm_operator* ops, int batch) {
  std::vector<int> ord(batch);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return ops[a].n > ops[b].n; });
  return ord;
}

// ------------------------------------------------------------------ large partial-DCT problems
// A batch splits into the problems of the persistent kernel and groups of equal n for the
// lockstep multi-pass solver, run one after the other on the caller's stream.
struct Split {
  std::vector<int> small;
  std::vector<std::pair<int64_t, std::vector<int>>> groups;
  bool any_large() const { return !groups.empty(); }
};
Split split_batch(const mfipm_operator* ops, int batch) {
  Split sp;
  for (int i = 0; i < batch; ++i) {
    if (!is_large_dct(ops[i])) {
      sp.small.push_back(i);
      continue;
    }
    auto it = std::find_if(sp.groups.begin(), sp.groups.end(), [&](auto& g) { return g.first == ops[i].n; });
    if (it == sp.groups.end()) sp.groups.push_back({ops[i].n, {i}});
    else it->second.push_back(i);
  }
  return sp;
}
size_t split_small_bytes(const mfipm_operator* ops, const Split& sp, const mfipm_params* p) {
  if (sp.small.empty()) return 0;
  std::vector<mfipm_operator> sub;
  for (int i : sp.small) sub.push_back(ops[i]);
  return align256(make_layout(sub.data(), (int)sub.size(), pcg_in_fp64(sub[0], p)).total);
}
size_t split_large_bytes(const Split& sp) {
  size_t b = 0;
  for (auto& g : sp.groups) b = std::max(b, large_dct_workspace_bytes(g.first, (int)g.second.size()));
  return b;
}
template <class T> std::vector<T> pick(const T* a, const std::vector<int>& idx) {
  std::vector<T> r;
  for (int i : idx) r.push_back(a ? a[i] : T{});
  return r;
}

// forward (gx == null) or backward solve of the large groups
int run_large_groups(const mfipm_operator* ops, const Split& sp, const double* const* b, const double* tau,
                     double* const* x, double* const* zs_out, const double* const* zs_in,
                     const double* const* gx, double* const* grad_b, double* grad_tau, const mfipm_params* p,
                     char* ws, size_t ws_bytes, mfipm_info* infos, cudaStream_t st) {
  for (auto& g : sp.groups) {
    const std::vector<int>& idx = g.second;
    const int R = (int)idx.size();
    std::vector<int64_t> ms;
    std::vector<const int64_t*> rows;
    for (int i : idx) {
      ms.push_back(ops[i].m);
      rows.push_back(ops[i].rows);
    }
    auto vb = pick(b, idx);
    auto vt = pick(tau, idx);
    auto vx = pick(x, idx);
    auto vz = pick(zs_out, idx);
    auto vzi = pick(zs_in, idx);
    auto vgx = pick(gx, idx);
    auto vgb = pick(grad_b, idx);
    std::vector<double> gt(R, 0.0);
    std::vector<mfipm_info> inf(R);
    LdCall c{};
    c.n = g.first;
    c.R = R;
    c.m = ms.data();
    c.rows = rows.data();
    c.b = vb.data();
    c.tau = tau ? vt.data() : nullptr;
    c.x = x ? vx.data() : nullptr;
    c.zs_out = zs_out ? vz.data() : nullptr;
    c.zs_in = zs_in ? vzi.data() : nullptr;
    c.gx = gx ? vgx.data() : nullptr;
    c.grad_b = grad_b ? vgb.data() : nullptr;
    c.grad_tau = gt.data();
    c.infos = inf.data();
    c.workspace = ws;
    c.ws_bytes = ws_bytes;
    c.prm = to_solve(p);
    c.stream = st;
    std::string msg;
    const int rc = gx ? large_dct_backward(c, &msg) : large_dct_solve(c, &msg);
    if (rc) return fail(rc, "%s", msg.c_str());
    for (int k = 0; k < R; ++k) {
      if (infos) infos[idx[k]] = inf[k];
      if (grad_tau && gx) grad_tau[idx[k]] = gt[k];
    }
  }
  return MFIPM_OK;
}

__device__ int g_gemm_err_word;
int* g_gemm_err_ptr() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_gemm_err_word) != cudaSuccess) return nullptr;
  return static_cast<int*>(p);
}

// ------------------------------------------------------------------ bf16 shared-A solver
int solve_shared_bf16(int batch, const mfipm_operator* ops, const double* const* b, const double* tau,
                      const mfipm_params* p, double* const* x, double* const* zs_out, void* workspace,
                      size_t ws_bytes, mfipm_info* infos, void* stream) {
  for (int i = 0; i < batch; ++i) {
    if (!(tau[i] > 0.0) || !isfinite(tau[i])) return fail(MFIPM_INVALID_ARG, "tau[%d] must be positive and finite", i);
    if (!b[i] || !x[i]) return fail(MFIPM_INVALID_ARG, "b[%d] or x[%d] is NULL", i, i);
  }
  if (p->centrality_correctors > 0)
    return fail(MFIPM_UNSUPPORTED, "multiple centrality correctors run on the persistent kernel only, not on the "
                "shared-A bf16 solver");
  size_t need = 0;
  int rc = mfipm_workspace_size(ops, batch, p, &need);
  if (rc) return rc;
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(MFIPM_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  if (ws_bytes < need) return fail(MFIPM_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  double* fro = reinterpret_cast<double*>(ws);
  mfipm_info* info_dev = reinterpret_cast<mfipm_info*>(ws + 256);
  const size_t off = 256 + ((sizeof(mfipm_info) * batch + 255) & ~(size_t)255) + 256;
  cudaError_t e = bf16_fro2(ops[0].A, ops[0].m, ops[0].n, ops[0].lda, fro, st);
  if (e) return cuda_fail(e, "norm of A");
  double fro2 = 0.0;
  if ((e = cudaMemcpyAsync(&fro2, fro, 8, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
    return cuda_fail(e, "norm of A");
  MrhsCall call{};
  call.m = ops[0].m;
  call.n = ops[0].n;
  call.lda = ops[0].lda;
  call.R = batch;
  call.A = ops[0].A;
  call.a_scale = ops[0].a_scale;
  // rho = ||A||_F^2 / n (reading R2) for the true matrix a_scale * A
  call.rho = fro2 * ops[0].a_scale * ops[0].a_scale / (double)ops[0].n;
  call.b = b;
  call.tau = tau;
  call.x = x;
  call.zs_out = zs_out;
  call.infos_dev = info_dev;
  call.workspace = ws + off;
  call.ws_bytes = ws_bytes - off;
  call.prm = to_solve(p);
  call.stream = st;
  int* err_dev = reinterpret_cast<int*>(ws + 64);
  if ((e = cudaMemsetAsync(err_dev, 0, 4, st))) return cuda_fail(e, "clear error word");
  call.err_dev = err_dev;
  call.resid_tc = g_resid_tc && !g_force_simple_gemm;
  const int m32 = (int)ops[0].m, n32 = (int)ops[0].n;
  if (tc_gemm_supported(m32, 2 * batch, n32) && tc_gemm_supported(n32, 2 * batch, m32) && !g_force_simple_gemm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    call.gemm = [](void* ctx, const void* Aop, const void* Bop, float* C, int rows, int N, int K, int splits,
                   cudaStream_t s2, int stages) {
      return tc_gemm(Aop, Bop, C, rows, N, K, splits, static_cast<int*>(ctx), s2, stages);
    };
    call.gemm_ctx = err_dev;
    call.splits1 = std::min(kMaxSplits, tc_gemm_splits(m32, n32, sms));
    call.splits2 = std::min(kMaxSplits, tc_gemm_splits(n32, m32, sms));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    call.stages1 = call.stages2 = 4;
    auto it = g_tune_gemm.find({ops[0].m, ops[0].n, batch});
    if (it != g_tune_gemm.end()) {
      call.splits1 = it->second.s1;
      call.splits2 = it->second.s2;
      call.stages1 = it->second.st1;
      call.stages2 = it->second.st2;
    }
  } else {
    call.gemm = gemm_simple;
    call.gemm_ctx = nullptr;
    call.splits1 = call.splits2 = 1;
  }
  std::string msg;
  rc = mrhs_solve(call, &msg);
  if (rc) return fail(rc, "%s", msg.c_str());
  int gemm_err = 0;
  if ((e = cudaMemcpyAsync(&gemm_err, err_dev, 4, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
    return cuda_fail(e, "read GEMM status");
  if (gemm_err) return fail(gemm_err, "tensor-core GEMM: a bounded mbarrier wait expired");
  std::vector<mfipm_info> tmp;
  if (!infos) {
    tmp.resize(batch);
    infos = tmp.data();
  }
  if ((e = cudaMemcpyAsync(infos, info_dev, sizeof(mfipm_info) * batch, cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st)))
    return cuda_fail(e, "read infos");
  for (int i = 0; i < batch; ++i)
    if (infos[i].status != MFIPM_OK) return infos[i].status;
  return MFIPM_OK;
}

// ------------------------------------------------------------------ fixed scratch
// Device scratch for mfipm_solve_noalloc, for callers that may not allocate device memory
// (see include/mfipm.h).  Every GPU that loads this library holds these bytes until the
// process exits.  In host code `g_noalloc_scratch` is only a stand-in for the symbol; its
// device address is obtained per device with cudaGetSymbolAddress.
constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
int noalloc_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(MFIPM_UNSUPPORTED, "device %d beyond the %d supported", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return MFIPM_OK;
}

int first_bad_status(const mfipm_info* infos, int batch) {
  for (int i = 0; i < batch; ++i)
    if (infos[i].status != MFIPM_OK) return infos[i].status;
  return MFIPM_OK;
}

// a batch with large partial-DCT problems: the rest by the persistent kernel, then the
// large groups, on one stream and one workspace
int solve_split(int batch, const mfipm_operator* ops, const double* const* b, const double* tau,
                const mfipm_params* p, double* const* x, double* const* zs_out, void* workspace, size_t ws_bytes,
                mfipm_info* infos, void* stream, const Split& sp) {
  for (int i = 0; i < batch; ++i) {
    if (!(tau[i] > 0.0) || !isfinite(tau[i])) return fail(MFIPM_INVALID_ARG, "tau[%d] must be positive and finite", i);
    if ((ops[i].m > 0 && !b[i]) || !x[i]) return fail(MFIPM_INVALID_ARG, "b[%d] or x[%d] is NULL", i, i);
    if (ops[i].kind != MFIPM_OP_PARTIAL_DCT) return fail(MFIPM_UNSUPPORTED, "a batch must use one operator kind");
  }
  if (p->precision != MFIPM_PREC_FP32_PCG)
    return fail(MFIPM_UNSUPPORTED, "the multi-pass partial-DCT solver (n >= its threshold) runs its PCG in float32 "
                "(precision=%d)", p->precision);
  if (p->centrality_correctors > 0 && !sp.groups.empty())
    return fail(MFIPM_UNSUPPORTED, "multiple centrality correctors run on the persistent kernel only, not on the "
                "multi-pass partial-DCT solver");
  const size_t small = split_small_bytes(ops, sp, p), need = small + split_large_bytes(sp);
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(MFIPM_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  if (ws_bytes < need) return fail(MFIPM_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  std::vector<mfipm_info> tmp;
  if (!infos) {
    tmp.resize(batch);
    infos = tmp.data();
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!sp.small.empty()) {
    const int ns = (int)sp.small.size();
    auto vo = pick(ops, sp.small);
    auto vb = pick(b, sp.small);
    auto vt = pick(tau, sp.small);
    auto vx = pick(x, sp.small);
    auto vz = pick(zs_out, sp.small);
    Prepared P;
    int rc = prepare(ns, vo.data(), vb.data(), vt.data(), p, vx.data(), zs_out ? vz.data() : nullptr, workspace,
                     small, P);
    if (rc) return rc;
    std::vector<mfipm_info> si(ns);
    std::vector<int> ord = cost_order(vo.data(), ns);
    rc = run(P, st, ns, si.data(), &ord);
    for (int k = 0; k < ns; ++k) infos[sp.small[k]] = si[k];
    if (rc && rc != MFIPM_NOT_CONVERGED && rc != MFIPM_NUMERIC) return rc;
  }
  int rc = run_large_groups(ops, sp, b, tau, x, zs_out, nullptr, nullptr, nullptr, nullptr, p,
                            static_cast<char*>(workspace) + small, ws_bytes - small, infos, st);
  if (rc) return rc;
  return first_bad_status(infos, batch);
}

int backward_persistent(int32_t batch, const mfipm_operator* ops, const double* const* b, const double* tau,
                   const double* const* x, const double* const* zs, const double* const* grad_x,
                   double* const* grad_b, double* grad_tau, double* const* grad_A, const mfipm_params* p,
                   void* workspace, size_t ws_bytes, mfipm_info* infos, void* stream) {
  Prepared P;
  int rc = prepare(batch, ops, b, tau, p, const_cast<double* const*>(x), nullptr, workspace, ws_bytes, P);
  if (rc) return rc;
  for (int i = 0; i < batch; ++i) {
    if (!zs[i] || !grad_x[i]) return fail(MFIPM_INVALID_ARG, "zs[%d] or grad_x[%d] is NULL", i, i);
    if (grad_A && grad_A[i] && ops[i].kind != MFIPM_OP_DENSE)
      return fail(MFIPM_UNSUPPORTED, "grad_A is defined for dense operators only (operator %d)", i);
    ProbDesc& d = P.desc[i];
    d.zs_in = zs[i];
    d.gx = grad_x[i];
    d.x_in = x[i];
    d.grad_b = grad_b ? grad_b[i] : nullptr;
    d.grad_A = grad_A ? grad_A[i] : nullptr;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(P.ws + P.lay.off_desc, P.desc.data(), sizeof(ProbDesc) * batch, cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cuda_fail(e, "upload descriptors");
  if ((e = cudaMemsetAsync(P.ws + P.lay.off_hdr, 0, 256, st)) != cudaSuccess) return cuda_fail(e, "clear header");
  if (P.dct) {
    if ((e = launch_twiddles(const_cast<double2*>(P.args.tw64), const_cast<float2*>(P.args.tw32),
                             const_cast<float4*>(P.args.twdf), P.args.log2_tw, st)) != cudaSuccess)
      return cuda_fail(e, "twiddle kernel");
    if ((e = launch_dct_setup(P.args.probs, batch, P.max_n, P.args.err, st)) != cudaSuccess)
      return cuda_fail(e, "setup kernel");
  }
  if (P.gen)
    for (auto& t : P.lay.gen_tabs)
      if ((e = launch_gen_twiddles(P.ws + t.second, t.first, st)) != cudaSuccess) return cuda_fail(e, "roots table");
  const int maxc = P.gen    ? max_active_ctas_bwd_dct_gen(P.max_n)
                   : P.haar ? max_active_clusters_bwd_haar(P.G, P.max_n)
                   : P.dct ? max_active_clusters_bwd_dct(P.G, P.max_n)
                           : max_active_clusters_bwd_dense(P.G, P.pcg64, P.max_n, P.max_m);
  if (maxc < 1) return fail(MFIPM_UNSUPPORTED, "no resident cluster of size %d fits this problem", P.G);
  const int clusters = std::min(maxc, batch);
  e = P.gen    ? launch_bwd_dct_gen(P.args, P.max_n, clusters, st)
      : P.haar ? launch_bwd_haar(P.G, P.args, P.max_n, clusters, st)
      : P.dct ? launch_bwd_dct(P.G, P.args, P.max_n, clusters, st)
              : launch_bwd_dense(P.G, P.pcg64, P.args, P.max_n, P.max_m, clusters, st);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  note_launches((P.dct ? 4 + (int64_t)P.lay.gen_tabs.size() : 0) + 1);
  std::vector<double> gt(batch);
  std::vector<mfipm_info> tmp;
  if (!infos) {
    tmp.resize(batch);
    infos = tmp.data();
  }
  int err = 0;
  if ((e = cudaMemcpyAsync(&err, P.args.err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(gt.data(), P.ws + P.lay.off_gtau, sizeof(double) * batch, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(infos, P.ws + P.lay.off_info, sizeof(mfipm_info) * batch, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
    return cuda_fail(e, "read results");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "backward");
  if (err == -1) return fail(MFIPM_INVALID_ARG, "rows must be distinct, ascending and inside [0, n)");
  if (err == -2) return fail(MFIPM_NUMERIC, "b contains a non-finite value");
  if (grad_tau)
    for (int i = 0; i < batch; ++i) grad_tau[i] = gt[i];
  return MFIPM_OK;
}

int apply_checked(int what, const mfipm_operator* op, const double* in, const double* b, double tau, double* out,
                  double* kkt, void* workspace, size_t ws_bytes, void* stream) {
  g_err.clear();
  int rc = validate_op(op, 0);
  if (rc) return rc;
  if (!in || (what < 2 && !out) || (what == 2 && (!kkt || (op->m > 0 && !b))))
    return fail(MFIPM_INVALID_ARG, "NULL vector argument");
  if (what == 2 && !(tau > 0.0 && isfinite(tau))) return fail(MFIPM_INVALID_ARG, "tau must be positive and finite");
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(MFIPM_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  std::string msg;
  rc = apply_operator(what, *op, in, b, tau, out, kkt, workspace, ws_bytes, static_cast<cudaStream_t>(stream), &msg);
  return rc ? fail(rc, "%s", msg.c_str()) : MFIPM_OK;
}

// ------------------------------------------------------------------ autotuner
// Persistent partial-DCT kernel: every (G, single-CTA limit) that fits the batch, timed by the
// solver kernel's CUDA events on the caller's problems (second of two runs).
int tune_dct(int batch, const mfipm_operator* ops, const double* const* b, const double* tau, const mfipm_params* p,
             double* const* x, void* workspace, size_t ws_bytes, mfipm_info* infos, cudaStream_t st,
             mfipm_tuning* t) {
  int64_t max_n = 0, min_n = INT64_MAX;
  for (int i = 0; i < batch; ++i) {
    max_n = std::max<int64_t>(max_n, ops[i].n);
    min_n = std::min<int64_t>(min_n, ops[i].n);
  }
  mfipm_params q = *p;
  q.cluster_size = 0;
  std::vector<mfipm_operator> vops(ops, ops + batch);
  const int G0 = pick_G(vops, &q, batch);
  const int64_t cm0 = std::min<int64_t>(16384, max_n / G0);
  std::vector<std::pair<int, int64_t>> cands{{G0, cm0}};
  for (int G = 1; G <= 16; G *= 2) {
    if (G < dct_min_G(max_n) || G > dct_max_G(min_n)) continue;
    for (int64_t cm : {2048, 4096, 8192, 16384}) {
      if (cm > std::min<int64_t>(16384, max_n / G) || (G == G0 && cm == cm0)) continue;
      if (G == 1 && cm != std::min<int64_t>(16384, max_n)) continue;  // one CTA each: the limit plays no part
      cands.push_back({G, cm});
    }
  }
  const std::vector<int> ord = cost_order(ops, batch);
  auto run_cfg = [&](int G, int64_t cm, int reps, double* ms) -> int {
    q.cluster_size = G;
    Prepared P;
    int rc = prepare(batch, ops, b, tau, &q, x, nullptr, workspace, ws_bytes, P);
    if (rc) return rc;
    P.cta_max_n = cm;
    const bool saved = g_timing;
    g_timing = true;
    for (int r = 0; r < reps && !rc; ++r) rc = run(P, st, batch, infos, &ord);
    g_timing = saved;
    *ms = g_last_ms;
    return rc;
  };
  double best = 1e300, dflt = -1.0;
  std::pair<int, int64_t> pick = cands[0];
  int timed = 0;
  for (size_t c = 0; c < cands.size(); ++c) {
    double ms = 0.0;
    if (run_cfg(cands[c].first, cands[c].second, 2, &ms) != MFIPM_OK) continue;  // skipped: did not solve
    ++timed;
    if (c == 0) dflt = ms;
    if (ms < best) {
      best = ms;
      pick = cands[c];
    }
  }
  if (!timed) return fail(MFIPM_NOT_CONVERGED, "autotune: no configuration solved the batch");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_dct[{max_n, ceil_log2i(batch)}] = TuneDct{pick.first, pick.second};
  }
  double ms = 0.0;
  const int rc = run_cfg(pick.first, pick.second, 1, &ms);  // x and infos from the chosen configuration
  if (t) {
    t->path = 1;
    t->candidates = timed;
    t->cluster_size = pick.first;
    t->cta_max_n = pick.second;
    t->best_ms = best;
    t->default_ms = dflt;
  }
  return rc;
}

// Shared bf16 A: split-K of T = A W and of Y = A^T T, each timed alone on its real shapes
// (median of 5), scratch operands carved from the caller's workspace.
int tune_gemm(int batch, const mfipm_operator* ops, void* workspace, size_t ws_bytes, cudaStream_t st,
              mfipm_tuning* t, int* s1_out, int* s2_out) {
  const int m = (int)ops[0].m, n = (int)ops[0].n, N = 2 * batch;
  *s1_out = *s2_out = 0;
  if (!tc_gemm_supported(m, N, n) || !tc_gemm_supported(n, N, m) || g_force_simple_gemm) return MFIPM_OK;
  char* ws = static_cast<char*>(workspace);
  const size_t wb = align256((size_t)N * n * 2), tb = align256((size_t)N * m * 2);
  const size_t cb = align256((size_t)kMaxSplits * N * std::max(m, n) * 4);
  if (wb + tb + cb > ws_bytes) return fail(MFIPM_INVALID_ARG, "autotune: workspace too small");
  void* W = ws;
  void* T = ws + wb;
  float* Cb = reinterpret_cast<float*>(ws + wb + tb);
  int* err = g_gemm_err_ptr();
  if (!err) return fail(MFIPM_CUDA, "no device error word");
  cudaError_t e;
  if ((e = cudaMemsetAsync(W, 0, wb + tb, st)) || (e = cudaMemsetAsync(err, 0, 4, st))) return cuda_fail(e, "autotune");
  cudaEvent_t ev[2];
  if ((e = cudaEventCreate(&ev[0])) || (e = cudaEventCreate(&ev[1]))) return cuda_fail(e, "autotune events");
  // the second GEMM reads A^T (n x m, K-major); A's own bytes viewed with that shape time the same
  auto time_one = [&](int rows, int K, const void* Bop, int s, int stg, double* ms) -> cudaError_t {
    std::vector<float> v;
    for (int r = 0; r < 6; ++r) {
      cudaError_t r2;
      if ((r2 = cudaEventRecord(ev[0], st)) || (r2 = tc_gemm(ops[0].A, Bop, Cb, rows, N, K, s, err, st, stg)) ||
          (r2 = cudaEventRecord(ev[1], st)) || (r2 = cudaEventSynchronize(ev[1])))
        return r2;
      float x = 0.f;
      cudaEventElapsedTime(&x, ev[0], ev[1]);
      if (r) v.push_back(x);
    }
    std::sort(v.begin(), v.end());
    *ms = v[v.size() / 2];
    return cudaSuccess;
  };
  double b1 = 1e300, b2 = 1e300, d1 = 0, d2 = 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int s1d = std::min(kMaxSplits, tc_gemm_splits(m, n, sms)), s2d = std::min(kMaxSplits, tc_gemm_splits(n, m, sms));
  int timed = 0, st1 = 4, st2 = 4;
  for (int stg = 4; stg >= 3 && !e; --stg) {  // 3 stages: two CTAs per SM at N <= 128
    for (int s = 1; s <= kMaxSplits; ++s) {  // every count: grid fill is not monotone in s
      double ms1 = 0, ms2 = 0;
      if ((e = time_one(m, n, W, s, stg, &ms1)) || (e = time_one(n, m, T, s, stg, &ms2))) break;
      timed += 2;
      if (stg == 4 && s == s1d) d1 = ms1;
      if (stg == 4 && s == s2d) d2 = ms2;
      if (ms1 < b1) { b1 = ms1; *s1_out = s; st1 = stg; }
      if (ms2 < b2) { b2 = ms2; *s2_out = s; st2 = stg; }
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e) return cuda_fail(e, "autotune GEMM");
  int herr = 0;
  if ((e = cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost))) return cuda_fail(e, "autotune GEMM status");
  if (herr) return fail(herr, "tensor-core GEMM: a bounded mbarrier wait expired");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_gemm[{ops[0].m, ops[0].n, batch}] = TuneGemm{*s1_out, *s2_out, st1, st2};
  }
  if (t) {
    t->path = 2;
    t->candidates = timed;
    t->splits1 = *s1_out;
    t->splits2 = *s2_out;
    t->stages1 = st1;
    t->stages2 = st2;
    t->best_ms = b1 + b2;
    t->default_ms = d1 + d2;
  }
  return MFIPM_OK;
}
}  // namespace

extern "C" {

int mfipm_params_default(mfipm_params* p) {
  if (!p) return fail(MFIPM_INVALID_ARG, "params is NULL");
  memset(p, 0, sizeof(*p));
  p->tol = 1e-10;
  p->max_iter = 100;
  p->tol_pcg = 1e-2;
  p->max_iter_pcg = 200;
  p->sigma1 = 0.1;
  p->sigma2 = 0.5;
  p->sigma3 = 0.8;
  p->alpha_bar = 0.5;
  p->alpha_tilde = 0.1;
  p->eta = 0.995;
  p->precision = MFIPM_PREC_FP32_PCG;
  p->equal_steps = 0;
  p->cluster_size = 0;
  p->outer = MFIPM_OUTER_DF;
  p->outer_f32_gap = 1e-8;
  return MFIPM_OK;
}

int mfipm_workspace_size(const mfipm_operator* ops, int32_t batch, const mfipm_params* p, size_t* bytes) {
  if (!ops || !bytes || batch < 1) return fail(MFIPM_INVALID_ARG, "NULL argument or batch < 1");
  int rc = validate_params(p);
  if (rc) return rc;
  for (int i = 0; i < batch; ++i)
    if ((rc = validate_op(&ops[i], i))) return rc;
  bool shared = false;
  if ((rc = check_shared_bf16(ops, batch, p, &shared))) return rc;
  if (shared) {
    *bytes = 256 + ((sizeof(mfipm_info) * batch + 255) & ~(size_t)255) + 256 + mrhs_workspace_bytes(ops[0].m, ops[0].n, batch);
    return MFIPM_OK;
  }
  const Split sp = split_batch(ops, batch);
  if (sp.any_large()) {
    *bytes = split_small_bytes(ops, sp, p) + split_large_bytes(sp);
    return MFIPM_OK;
  }
  *bytes = make_layout(ops, batch, pcg_in_fp64(ops[0], p)).total;
  return MFIPM_OK;
}

int mfipm_solve(const mfipm_operator* op, const double* b, double tau, const mfipm_params* p, double* x,
                double* zs_out, void* workspace, size_t ws_bytes, mfipm_info* info, void* stream) {
  g_err.clear();
  lockstep_stats_reset();
  const double* bb[1] = {b};
  double* xx[1] = {x};
  double* zz[1] = {zs_out};
  double tt[1] = {tau};
  if (op && p && op->kind == MFIPM_OP_DENSE && op->a_dtype == MFIPM_A_BF16 && p->precision == MFIPM_PREC_BF16_A) {
    int rc = validate_params(p);
    if (rc || (rc = validate_op(op, 0))) return rc;
    return solve_shared_bf16(1, op, bb, tt, p, xx, zs_out ? zz : nullptr, workspace, ws_bytes, info, stream);
  }
  if (op && p && is_large_dct(*op)) {
    int rc = validate_params(p);
    if (rc || (rc = validate_op(op, 0))) return rc;
    return solve_split(1, op, bb, tt, p, xx, zs_out ? zz : nullptr, workspace, ws_bytes, info, stream,
                       split_batch(op, 1));
  }
  Prepared P;
  int rc = prepare(1, op, bb, tt, p, xx, zs_out ? zz : nullptr, workspace, ws_bytes, P);
  if (rc) return rc;
  mfipm_info tmp;
  return run(P, static_cast<cudaStream_t>(stream), 1, info ? info : &tmp, nullptr);
}

int mfipm_solve_noalloc(const mfipm_operator* op, const double* b, double tau, const mfipm_params* p, double* x,
                        double* zs_out, mfipm_info* info, void* stream) {
  g_err.clear();
  size_t need = 0;
  int rc = mfipm_workspace_size(op, 1, p, &need);
  if (rc) return rc;
  if (need > kNoallocScratchBytes)
    return fail(MFIPM_INVALID_ARG,
                "mfipm_solve_noalloc: this problem needs %zu bytes of scratch, above the fixed %zu bytes; "
                "use mfipm_solve with a caller workspace",
                need, kNoallocScratchBytes);
  void* ws = nullptr;
  if ((rc = noalloc_scratch(&ws))) return rc;
  // the same dispatch as mfipm_solve (shared-A bf16, multi-pass partial DCT, persistent kernel),
  // whose workspace need is the one checked above
  return mfipm_solve(op, b, tau, p, x, zs_out, ws, kNoallocScratchBytes, info, stream);
}

int mfipm_solve_batched(int32_t batch, const mfipm_operator* ops, const double* const* b, const double* tau,
                        const mfipm_params* p, double* const* x, double* const* zs_out, void* workspace,
                        size_t ws_bytes, mfipm_info* infos, void* stream) {
  g_err.clear();
  lockstep_stats_reset();
  {
    int rc = validate_params(p);
    if (rc) return rc;
    if (batch < 1 || !ops || !b || !tau || !x) return fail(MFIPM_INVALID_ARG, "NULL argument array or batch < 1");
    for (int i = 0; i < batch; ++i)
      if ((rc = validate_op(&ops[i], i))) return rc;
    bool shared = false;
    if ((rc = check_shared_bf16(ops, batch, p, &shared))) return rc;
    if (shared) return solve_shared_bf16(batch, ops, b, tau, p, x, zs_out, workspace, ws_bytes, infos, stream);
    const Split sp = split_batch(ops, batch);
    if (sp.any_large()) return solve_split(batch, ops, b, tau, p, x, zs_out, workspace, ws_bytes, infos, stream, sp);
  }
  Prepared P;
  int rc = prepare(batch, ops, b, tau, p, x, zs_out, workspace, ws_bytes, P);
  if (rc) return rc;
  std::vector<mfipm_info> tmp;
  if (!infos) {
    tmp.resize(batch);
    infos = tmp.data();
  }
  std::vector<int> ord = cost_order(ops, batch);
  return run(P, static_cast<cudaStream_t>(stream), batch, infos, &ord);
}

int mfipm_backward(int32_t batch, const mfipm_operator* ops, const double* const* b, const double* tau,
                   const double* const* x, const double* const* zs, const double* const* grad_x,
                   double* const* grad_b, double* grad_tau, double* const* grad_A, const mfipm_params* p,
                   void* workspace, size_t ws_bytes, mfipm_info* infos, void* stream) {
  g_err.clear();
  lockstep_stats_reset();
  if (!zs || !grad_x) return fail(MFIPM_INVALID_ARG, "zs and grad_x are required");
  if (batch < 1 || !ops || !b || !tau || !x) return fail(MFIPM_INVALID_ARG, "NULL argument array or batch < 1");
  int rc = validate_params(p);
  if (rc) return rc;
  for (int i = 0; i < batch; ++i)
    if ((rc = validate_op(&ops[i], i))) return rc;
  const Split sp = split_batch(ops, batch);
  if (!sp.any_large())
    return backward_persistent(batch, ops, b, tau, x, zs, grad_x, grad_b, grad_tau, grad_A, p, workspace, ws_bytes,
                               infos, stream);
  for (int i = 0; i < batch; ++i) {
    if (!zs[i] || !grad_x[i] || !b[i] || !x[i]) return fail(MFIPM_INVALID_ARG, "argument %d is NULL", i);
    if (ops[i].kind != MFIPM_OP_PARTIAL_DCT) return fail(MFIPM_UNSUPPORTED, "a batch must use one operator kind");
    if (grad_A && grad_A[i]) return fail(MFIPM_UNSUPPORTED, "grad_A is defined for dense operators only (operator %d)", i);
  }
  if (p->precision != MFIPM_PREC_FP32_PCG)
    return fail(MFIPM_UNSUPPORTED, "the multi-pass partial-DCT solver (n >= its threshold) runs its PCG in float32 "
                "(precision=%d)", p->precision);
  if (p->centrality_correctors > 0 && !sp.groups.empty())
    return fail(MFIPM_UNSUPPORTED, "multiple centrality correctors run on the persistent kernel only, not on the "
                "multi-pass partial-DCT solver");
  const size_t small = split_small_bytes(ops, sp, p), need = small + split_large_bytes(sp);
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(MFIPM_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  if (ws_bytes < need) return fail(MFIPM_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  std::vector<mfipm_info> tmp;
  if (!infos) {
    tmp.resize(batch);
    infos = tmp.data();
  }
  if (!sp.small.empty()) {
    const int ns = (int)sp.small.size();
    auto vo = pick(ops, sp.small);
    auto vb = pick(b, sp.small);
    auto vt = pick(tau, sp.small);
    auto vx = pick(x, sp.small);
    auto vz = pick(zs, sp.small);
    auto vg = pick(grad_x, sp.small);
    auto vgb = pick(grad_b, sp.small);
    std::vector<double> gt(ns, 0.0);
    std::vector<mfipm_info> si(ns);
    rc = backward_persistent(ns, vo.data(), vb.data(), vt.data(), vx.data(), vz.data(), vg.data(),
                             grad_b ? vgb.data() : nullptr, gt.data(), nullptr, p, workspace, small, si.data(), stream);
    if (rc) return rc;
    for (int k = 0; k < ns; ++k) {
      infos[sp.small[k]] = si[k];
      if (grad_tau) grad_tau[sp.small[k]] = gt[k];
    }
  }
  return run_large_groups(ops, sp, b, tau, nullptr, nullptr, zs, grad_x, grad_b, grad_tau, p,
                          static_cast<char*>(workspace) + small, ws_bytes - small, infos,
                          static_cast<cudaStream_t>(stream));
}


int mfipm_apply_A(const mfipm_operator* op, const double* x, double* y, void* workspace, size_t ws_bytes,
                  void* stream) {
  return apply_checked(0, op, x, nullptr, 0.0, y, nullptr, workspace, ws_bytes, stream);
}
int mfipm_apply_At(const mfipm_operator* op, const double* y, double* x, void* workspace, size_t ws_bytes,
                   void* stream) {
  return apply_checked(1, op, y, nullptr, 0.0, x, nullptr, workspace, ws_bytes, stream);
}
int mfipm_kkt_residual(const mfipm_operator* op, const double* b, double tau, const double* x, void* workspace,
                       size_t ws_bytes, double* out, void* stream) {
  return apply_checked(2, op, x, b, tau, nullptr, out, workspace, ws_bytes, stream);
}

int mfipm_autotune(int32_t batch, const mfipm_operator* ops, const double* const* b, const double* tau,
                   const mfipm_params* p, double* const* x, void* workspace, size_t ws_bytes, mfipm_info* infos,
                   mfipm_tuning* tuning, void* stream) {
  g_err.clear();
  if (tuning) memset(tuning, 0, sizeof(*tuning));
  int rc = validate_params(p);
  if (rc) return rc;
  if (batch < 1 || !ops || !b || !tau || !x) return fail(MFIPM_INVALID_ARG, "NULL argument array or batch < 1");
  for (int i = 0; i < batch; ++i)
    if ((rc = validate_op(&ops[i], i))) return rc;
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(MFIPM_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  size_t need = 0;
  if ((rc = mfipm_workspace_size(ops, batch, p, &need))) return rc;
  if (ws_bytes < need) return fail(MFIPM_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<mfipm_info> tmp;
  if (!infos) {
    tmp.resize(batch);
    infos = tmp.data();
  }
  bool shared = false;
  if ((rc = check_shared_bf16(ops, batch, p, &shared))) return rc;
  if (shared) {
    int s1 = 0, s2 = 0;
    if ((rc = tune_gemm(batch, ops, workspace, ws_bytes, st, tuning, &s1, &s2))) return rc;
    return solve_shared_bf16(batch, ops, b, tau, p, x, nullptr, workspace, ws_bytes, infos, stream);
  }
  const Split sp = split_batch(ops, batch);
  if (ops[0].kind != MFIPM_OP_PARTIAL_DCT || sp.any_large() || p->cluster_size != 0 || needs_gen(ops, batch))
    return mfipm_solve_batched(batch, ops, b, tau, p, x, nullptr, workspace, ws_bytes, infos, stream);
  return tune_dct(batch, ops, b, tau, p, x, workspace, ws_bytes, infos, st, tuning);
}

int mfipm_clear_tuning(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_dct.clear();
  g_tune_gemm.clear();
  return MFIPM_OK;
}

const char* mfipm_last_error(void) { return g_err.c_str(); }

int mfipm_set_timing(int32_t enable) {
  g_timing = enable != 0;
  g_last_ms = -1.0f;
  large_dct_set_timing(enable != 0);
  return MFIPM_OK;
}

double mfipm_last_kernel_ms(void) { return (double)g_last_ms; }

int mfipm_last_operator_stats(double* ms, double* bytes, int64_t* products, int64_t* launches) {
  if (!ms || !bytes || !products || !launches) return fail(MFIPM_INVALID_ARG, "NULL output");
  large_dct_timing(ms, bytes, products, launches);
  return MFIPM_OK;
}

int mfipm_fp32_fma_peak(double* tflops, void* stream) {
  g_err.clear();
  if (!tflops) return fail(MFIPM_INVALID_ARG, "tflops is NULL");
  const cudaError_t e = measure_fp32_fma_peak(tflops, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MFIPM_OK : cuda_fail(e, "fp32 FMA probe");
}

int mfipm_set_gemm_mode(int32_t tensor_cores) {
  g_force_simple_gemm = tensor_cores == 0;
  return MFIPM_OK;
}

int mfipm_set_residual_mode(int32_t tensor_cores) {
  g_resid_tc = tensor_cores != 0;
  return MFIPM_OK;
}

int mfipm_set_large_dct_threshold(int64_t n) {
  if (n < kLdMinN) return fail(MFIPM_INVALID_ARG, "threshold below the multi-pass minimum %lld", (long long)kLdMinN);
  g_large_dct_min_n = std::min<int64_t>(n, 2 * kDctMaxN);
  return MFIPM_OK;
}

int mfipm_gemm_bf16(const void* Aop, const void* Bop, float* C, int32_t rows, int32_t N, int32_t K, int32_t splits,
                    int32_t tensor_cores, void* stream) {
  g_err.clear();
  if (!Aop || !Bop || !C || rows < 1 || N < 1 || K < 1 || splits < 1 || splits > kMaxSplits)
    return fail(MFIPM_INVALID_ARG, "mfipm_gemm_bf16: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (tensor_cores) {
    if (!tc_gemm_supported(rows, N, K)) return fail(MFIPM_UNSUPPORTED, "tensor-core GEMM needs N <= 256, K % 8 == 0");
    if (tensor_cores != 1 && tensor_cores != 3 && tensor_cores != 4)
      return fail(MFIPM_INVALID_ARG, "mfipm_gemm_bf16: tensor_cores must be 0, 1, 3 or 4");
    int* err_dev = g_gemm_err_ptr();  // a static device word: the call allocates nothing
    if (!err_dev) return fail(MFIPM_CUDA, "no device error word");
    if ((e = cudaMemsetAsync(err_dev, 0, 4, st))) return cuda_fail(e, "clear error word");
    if ((e = tc_gemm(Aop, Bop, C, rows, N, K, splits, err_dev, st, tensor_cores == 3 ? 3 : 4)))
      return cuda_fail(e, "tc_gemm");
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, err_dev, 4, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
      return cuda_fail(e, "tc_gemm status");
    if (herr) return fail(herr, "tensor-core GEMM: a bounded mbarrier wait expired");
    return MFIPM_OK;
  }
  if (splits != 1) return fail(MFIPM_INVALID_ARG, "the CUDA-core GEMM has no split-K");
  if ((e = gemm_simple(nullptr, Aop, Bop, C, rows, N, K, 1, st, 0))) return cuda_fail(e, "gemm_simple");
  if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "gemm_simple");
  return MFIPM_OK;
}

}  // extern "C"
