// C ABI of libhmc (include/hmc.h): handle life cycle, uploads, and the
// orchestration of the fused log-posterior/gradient pass, the split-K
// reduction + leapfrog update, and the momentum / accept / select kernels.
// One HMC iteration (Sec. 1.1: draw eta, L leapfrog updates, accept test) is
// captured once as a CUDA graph and replayed `iters` times; the iteration
// index the generator needs lives in device memory, so every replay is the
// same graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

using namespace hmc;

namespace {

thread_local std::string g_last_error;

hmc_status fail(hmc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define HMC_CUDA(call)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? HMC_ENOMEM : HMC_ECUDA,                             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                   \
    }                                                                                                   \
  } while (0)

#define HMC_TRY(expr)            \
  do {                           \
    hmc_status s_ = (expr);      \
    if (s_ != HMC_OK) return s_; \
  } while (0)

int dtype_bytes(int t) { return t == HMC_F64 ? 8 : t == HMC_F32 ? 4 : t == HMC_BF16 ? 2 : 1; }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct StateSet {
  void* beta = nullptr;
  void* eta = nullptr;
  void* grad = nullptr;
  void* beta0 = nullptr;
  void* grad0 = nullptr;
};

struct Problem {
  int64_t n = 0;
  int32_t p = 0, p_pad = 0, K = 0;
  int32_t Km1 = 0;     // free coefficient rows per chain the kernels see (K - 1, or K unconstrained)
  int32_t ku = 0;      // rows per chain of the user's beta layout (Km1, or K with the masked row)
  int32_t zlogit = 1;  // class K is the implied zero logit (identifiable layouts)
  void* X = nullptr;
  int32_t* y = nullptr;
  float* xscale = nullptr;
  // fused-pass configuration
  int S = 1, BM = 32, CR = 8, NT = 32, NWL = 1, NSTAGE = 2, PC = 32, nclusters = 1, ct_launch = 1, group_chains = 1;
  size_t smem = 0;
  int64_t ntiles = 0;
  void* gpart = nullptr;
  double* lpart = nullptr;
  StateSet cs, us;  // chain state (hmc_sample) and user-call scratch
  double* logk = nullptr;  // [2][max_chains]: chain state, user scratch
  double* logk0 = nullptr;
  double* h0 = nullptr;
  double* scal = nullptr;  // [max_chains][nblk][2]
  unsigned int* tickets = nullptr;  // [max_chains] + 1 (select)
  int* accept = nullptr;
  void* stats = nullptr;
  int64_t* iter = nullptr;  // [3]: global iteration, local iteration, generator seed
  int nblk = 1;
  int glanes = 1;           // lanes sharing one coefficient's split-K sum in the reduction
  int64_t state_elems = 0;  // max_chains * Km1 * p_pad
  // tensor-core engines
  int engine = 1;           // 1 CUDA-core fused kernel, 2 tensor-core fused kernel, 3 tensor-core two-pass,
                            // 4 CUDA-core two-pass
  TcPlan tp{};
  Tc2Plan tp2{};            // engine 3
  void* rbuf = nullptr;     // engines 3, 4: residuals written by the first pass, read by the second
  void* spart = nullptr;    // engine 3: partial logits of first-pass units split over two CTAs;
                            // engine 4: partial logits of the first pass's feature splits
  int fs = 1;               // engine 4: feature splits of the first pass
  int* sflag = nullptr;     // engine 3: their ready flags
  void* bbf = nullptr;      // BF16 coefficient operand boxes [p_pad / 64][2N x 128 B] (hi, lo terms)
  int nlparts = 0;          // log-likelihood partials reduced per chain
};

struct FusedTimer {
  std::vector<cudaEvent_t> ev;   // pairs
  std::vector<cudaEvent_t> mid;  // per pair: end of the first pass (two-pass engine), else unused
  std::vector<char> has_mid;
  size_t used = 0;
};

}  // namespace

struct hmc_ctx {
  int xt = HMC_F32, st = HMC_F32, prior_kind = 0, layout = HMC_LAYOUT_FREE;
  double prior_scale = 1.0;
  int max_chains = 1, engine = 0;
  long long spin_limit = 1ll << 22;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture / replay
  std::vector<Problem> probs;
  int* err_d = nullptr;
  int chains_init = 0;  // chains whose state has been initialised
  double* temps_d = nullptr;
  int64_t temps_cap = 0;
  void* staging[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t staging_cap[4] = {0, 0, 0, 0};
  bool timing = false;
  int timing_period = 1;    // events around every timing_period-th fused launch
  int64_t timing_seq = 0;   // fused launches issued since timing was enabled
  double timing_ms = 0.0;
  double timing_first_ms = 0.0;   // two-pass engine: the first pass's share of timing_ms
  int64_t timing_launches = 0;
  FusedTimer timer;
  std::string desc;
  int64_t chain_size = 0;
  int tile[4] = {0, 0, 0, 0};
  bool inject_timeout = false;  // HMC_FAULT=timeout at creation: first fused launch times out
  // One fused launch for every problem of a batch handle (CUDA-core engine).
  bool batched = false;
  int b_S = 1, b_NT = 32, b_NWL = 1, b_CT = 1, b_total_clusters = 0;
  size_t b_smem = 0;
  LpgArgs* b_table = nullptr;   // device [2][nprob]: chain state, user scratch
  int* b_first = nullptr;       // device [nprob + 1] first cluster of each problem
  // The same for the tensor-core engine (BF16 / FP8 storage).
  bool tc_batched = false;
  void* tb_table = nullptr;     // device TcArgs [nprob]
  void* tb_beta = nullptr;      // device coefficient-box jobs [2][nprob]: chain state, user scratch
  int64_t tb_max_elems = 0;     // largest N x p_pad of the operand boxes
  // Cached graph of one HMC iteration and the parameters baked into it.
  cudaGraphExec_t gexec = nullptr;
  int g_chains = 0, g_L = 0, g_thin = 0;
  double g_eps = 0.0;
  const void* g_samples = nullptr;
  bool g_temps = false, g_timing = false;
  int g_period = 1;
  const double* g_temps_ptr = nullptr;
  cudaStream_t g_stream = nullptr;
  size_t g_pairs = 0;
  std::vector<cudaEvent_t> g_events;  // timing events baked into the cached graph
  // Graphs of hmc_logpost_grad (slot 0) and hmc_leapfrog (slot 1) calls on
  // device buffers: captured when the same call (chains, buffers, L, eps,
  // stream) comes twice in a row and replayed while it keeps coming, so that a
  // call costs one graph launch instead of one launch per kernel.
  struct CallGraph {
    std::vector<uint64_t> key;
    bool seen = false;
    cudaGraphExec_t exec = nullptr;
  } cg[2];
};

namespace {

size_t state_bytes(const hmc_ctx* h) { return size_t(dtype_bytes(h->st)); }

hmc_status grow_staging(hmc_ctx* h, int slot, size_t bytes, void** out) {
  if (h->staging_cap[slot] < bytes) {
    if (h->staging[slot]) cudaFree(h->staging[slot]);
    h->staging[slot] = nullptr;
    h->staging_cap[slot] = 0;
    HMC_CUDA(cudaMalloc(&h->staging[slot], bytes));
    h->staging_cap[slot] = bytes;
  }
  *out = h->staging[slot];
  return HMC_OK;
}

// Device view of a user input buffer (copied to staging when on the host).
hmc_status dev_in(hmc_ctx* h, int slot, const void* user, size_t bytes, const void** dev) {
  if (!user || is_device_ptr(user)) {
    *dev = user;
    return HMC_OK;
  }
  void* d = nullptr;
  HMC_TRY(grow_staging(h, slot, bytes, &d));
  HMC_CUDA(cudaMemcpyAsync(d, user, bytes, cudaMemcpyHostToDevice, h->stream));
  *dev = d;
  return HMC_OK;
}

// Device destination for a user output buffer; *host says a copy-back is needed.
hmc_status dev_out(hmc_ctx* h, int slot, void* user, size_t bytes, void** dev, bool* host) {
  *host = false;
  if (!user || is_device_ptr(user)) {
    *dev = user;
    return HMC_OK;
  }
  *host = true;
  return grow_staging(h, slot, bytes, dev);
}

hmc_status check_device_error(hmc_ctx* h) {
  int e = 0;
  HMC_CUDA(cudaMemcpyAsync(&e, h->err_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  if (e) {
    HMC_CUDA(cudaMemsetAsync(h->err_d, 0, sizeof(int), h->stream));
    // A launch that gave up may have left a split unit's flag raised.
    for (Problem& P : h->probs)
      if (P.sflag) HMC_CUDA(cudaMemsetAsync(P.sflag, 0, size_t(P.tp2.gridA) * sizeof(int), h->stream));
    HMC_CUDA(cudaStreamSynchronize(h->stream));
    if (e & (ERR_TIMEOUT_STAGE | ERR_TIMEOUT_EXCHANGE | ERR_TIMEOUT_SLOT | ERR_TIMEOUT_MMA))
      return fail(HMC_ETIMEOUT, "a bounded device wait ran out (error bits " + std::to_string(e) + ")");
    if (e & (ERR_BAD_LABEL | ERR_NONFINITE_X))
      return fail(HMC_ENONFINITE, "label outside [0, K) or non-finite X (error bits " + std::to_string(e) + ")");
    return fail(HMC_ECUDA, "device error bits " + std::to_string(e));
  }
  return HMC_OK;
}

// ------------------------------------------------------------- configuration
// Chains per launch when at most gmax fit one launch: the fewest launches, with
// the chains spread evenly over them (16 chains at gmax 14 run as 8 + 8, not 14 + 2;
// every launch streams X once, so a small remainder group costs a full pass).
int balanced_group(int chains, int gmax) {
  const int launches = (chains + gmax - 1) / gmax;
  return (chains + launches - 1) / launches;
}

// Tensor-core plan: the largest chain group whose coefficient columns fit TMEM
// next to the cluster's gradient slice (evened out over the launches it takes),
// then the cluster size that keeps the most SMs busy.
hmc_status choose_tc(hmc_ctx* h, Problem& P, bool* ok) {
  *ok = false;
  if (P.Km1 > 32) return HMC_OK;   // the softmax maps one (row, chain) task to a warp, class <-> lane
  int dev = 0, smem_max = 0;
  HMC_CUDA(cudaGetDevice(&dev));
  HMC_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int best_g = 0, best_sms = 0;
  TcPlan best{};
  int best_nst = 0;
  size_t best_smem = 0;
  int best_maxclu = 0;
  for (int S : {16, 8, 4, 2, 1}) {
    if (h->tile[0] && S != h->tile[0]) continue;
    int g_even = 0;
    for (int g = h->max_chains; g >= 1; --g) {
      if (g_even && g > g_even) continue;
      TcPlan pl;
      if (!tc_plan(P.p, g * P.Km1, S, &pl)) continue;
      // Exchange depth (partial-logit slots and R buffers) and sweep lookahead:
      // 2 when TMEM holds a second logit accumulator, unless overridden by
      // opts.tile[1] / tile[2]; the deepest ring that fits shared memory next
      // to them, falling back to depth 1 when depth 2 leaves no room.
      const int d_want = h->tile[1] ? h->tile[1] : (pl.nz >= 2 ? 2 : 1);
      const int la_want = h->tile[2] ? h->tile[2] : (pl.nz >= 2 ? 2 : 1);
      int nst = 0;
      size_t smem = 0;
      for (int d = d_want; d >= 1 && !nst; --d) {
        if (h->tile[1] && d != h->tile[1]) continue;
        pl.slots = pl.rbufs = d;
        // Sweep 2 of tile u waits for the R rows of u, which need every CTA's
        // sweep 2 of tile u - d: lookahead below nz + 2d - 1 keeps that chain acyclic.
        pl.la = std::max(1, std::min(d == d_want ? la_want : 1, pl.nz + 2 * d - 2));
        for (int s = 6; s >= 2; --s) {
          if (h->tile[3] && s != h->tile[3]) continue;
          // At least half of an SM's shared memory: one CTA per SM, so no CTA
          // ever waits for TMEM held by a CTA of another cluster.
          const size_t sm = std::max(tc_smem_bytes(pl, s, g, h->xt == HMC_FP8E4M3), size_t(116 * 1024));
          if (sm <= size_t(smem_max)) {
            nst = s;
            smem = sm;
            break;
          }
        }
      }
      if (!nst) continue;
      HMC_CUDA(tc_prepare(smem, S, h->xt == HMC_FP8E4M3));
      int maxclu = 0;
      if (tc_max_active_clusters(smem, S, h->xt == HMC_FP8E4M3, &maxclu) != cudaSuccess) {
        cudaGetLastError();
        maxclu = 0;
      }
      if (maxclu < 1) continue;
      if (!g_even) {
        // Largest group that fits: plan again at the even split if it is smaller.
        g_even = balanced_group(h->max_chains, g);
        if (g_even < g) continue;
      }
      const int sms = maxclu * S;
      if (g > best_g || (g == best_g && sms > best_sms)) {
        best_g = g;
        best_sms = sms;
        best = pl;
        best_nst = nst;
        best_smem = smem;
        best_maxclu = maxclu;
      }
      break;  // largest group for this S found
    }
  }
  if (!best_g) return HMC_OK;
  P.engine = 2;
  P.tp = best;
  P.group_chains = best_g;
  P.ct_launch = best_g * P.Km1;
  P.S = best.S;
  P.PC = best.PC;
  P.p_pad = best.S * best.PC;
  P.BM = 128;
  P.CR = 128;
  P.NT = tc_threads(h->xt == HMC_FP8E4M3);
  P.NSTAGE = best_nst;
  P.smem = best_smem;
  P.ntiles = (P.n + 127) / 128;
  P.nclusters = int(std::max<int64_t>(1, std::min<int64_t>(best_maxclu, P.ntiles)));
  HMC_CUDA(tc_prepare(P.smem, P.S, h->xt == HMC_FP8E4M3));
  *ok = true;
  return HMC_OK;
}

hmc_status setup_problem(hmc_ctx* h, Problem& P, const void* X, int x_dtype, const int32_t* y) {
  const int xb = dtype_bytes(h->xt);
  bool tc_ok = false;
  if ((h->xt == HMC_BF16 || h->xt == HMC_FP8E4M3) && (h->engine == 0 || h->engine == 2) && P.n > 0)
    HMC_TRY(choose_tc(h, P, &tc_ok));
  if (h->engine == 2 && !tc_ok)
    return fail(HMC_EUNSUPPORTED, "the tensor-core engine needs BF16 or FP8 storage of X, n > 0 and chains * (K-1) "
                                  "columns that fit TMEM next to the cluster's gradient slice");
  // Two-pass tensor-core engine: on request, or by default for BF16 / FP8 X:
  // always for a single problem (its two passes stream X at a higher rate than
  // the fused pass's tile pipeline: n=5e4 p=1e4 K=20, 4 chains, BF16 402 against
  // 614 us per gradient, FP8 806 against 1017 us), and, BF16, in a batch when the
  // fused engine cannot take every chain in one launch (each launch would stream
  // X again) or cannot run the problem.
  const bool single = h->probs.size() == 1;
  const bool tcx = h->xt == HMC_BF16 || h->xt == HMC_FP8E4M3;
  const bool want2 = tcx && P.n > 0 && P.Km1 <= 32 &&
                     (h->engine == 3 ||
                      (h->engine == 0 && !h->tile[0] &&
                       (single || (h->xt == HMC_BF16 && (!tc_ok || P.group_chains < h->max_chains)))));
  if (want2) {
    int dev = 0, nsm = 0, smem_max = 0;
    HMC_CUDA(cudaGetDevice(&dev));
    HMC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HMC_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    Tc2Plan p2;
    if (tc2_plan(P.n, P.p, P.Km1, h->max_chains, nsm, smem_max, h->engine == 3 ? h->tile[0] : 0, &p2)) {
      HMC_CUDA(tc2_prepare());
      P.engine = 3;
      P.tp2 = p2;
      P.group_chains = h->max_chains;
      P.ct_launch = h->max_chains * P.Km1;
      P.S = 1;
      P.PC = p2.p_pad;
      P.p_pad = p2.p_pad;
      P.BM = 128;
      P.CR = 128;
      P.NT = tc2_threads(h->xt == HMC_FP8E4M3);
      P.NSTAGE = p2.nstA;
      P.smem = p2.smemA;
      P.ntiles = (P.n + 127) / 128;
      P.nclusters = p2.Q;           // partial gradient slices reduced per gradient
      tc_ok = true;
    }
  }
  if (h->engine == 3 && P.engine != 3)
    return fail(HMC_EUNSUPPORTED, "the two-pass tensor-core engine needs BF16 or FP8 storage of X, n > 0, at most 32 free "
                                  "classes per chain and (opts.tile[0]) row tiles per unit that fit TMEM");
  if (!tc_ok) {
    if (h->tile[1] || h->tile[2])
      return fail(HMC_EINVAL, "tile[1] and tile[2] must be 0 on the CUDA-core engines");
    const int maxct = simt_max_ct(h->xt);
    int dev = 0, nsm = 0;
    HMC_CUDA(cudaGetDevice(&dev));
    HMC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // Fused CUDA-core pass first (X read once); two CUDA-core passes where it
    // has no tile (wide problems with many classes: the coefficient slice and
    // the ring of row tiles do not fit one cluster) or more classes per chain
    // than it handles.
    SimtTile tc{};
    if (h->engine != 4 && P.Km1 <= maxct) {
      P.group_chains = balanced_group(h->max_chains, std::max(1, std::min(h->max_chains, maxct / P.Km1)));
      P.ct_launch = P.group_chains * P.Km1;
      P.ntiles = (P.n + kSimtRows - 1) / kSimtRows;
      HMC_CUDA(simt_choose(h->xt, P.ct_launch, P.p, P.ntiles, h->tile[0], h->tile[3], 0, &tc));
    }
    // By default also for a single problem with many coefficient columns, where
    // its class-split passes beat the fused pass's register-held columns
    // (measured: all chains' columns C >= 14 at p >= 2048, or C >= 19, on X of
    // at least 4e6 elements; e.g. n=2e4 p=1e4 K=15, one chain: 619 against 985 us).
    const int64_t c_all = int64_t(h->max_chains) * P.Km1;
    const bool wide = h->probs.size() == 1 && P.n * P.p >= 4000000 &&
                      (c_all >= 19 || (c_all >= 14 && P.p >= 2048));
    const bool two = (h->xt == HMC_F32 || h->xt == HMC_F64) && P.n > 0 && P.Km1 <= simt2_max_c() &&
                     (h->engine == 4 || (h->engine == 0 && !h->tile[0] && !h->tile[3] && (!tc.S || wide)));
    if (two) {
      P.engine = 4;
      P.group_chains = balanced_group(h->max_chains, std::max(1, std::min(h->max_chains, simt2_max_c() / P.Km1)));
      P.ct_launch = P.group_chains * P.Km1;
      P.S = 1;
      P.p_pad = (P.p + 3) / 4 * 4;
      P.PC = P.p_pad;
      P.BM = 1;
      P.CR = 1;
      P.NT = 256;
      P.NSTAGE = 0;
      P.smem = 0;
      P.ntiles = P.n;
      P.nclusters = simt2_row_ranges(P.n, P.p_pad, P.ct_launch, nsm);   // partial gradient slices of the second pass
      P.fs = simt2_feature_splits(P.n, P.p_pad, nsm);
      HMC_CUDA(simt2_prepare(h->xt));
    } else if (h->engine == 4) {
      return fail(HMC_EUNSUPPORTED, "the two-pass CUDA-core engine needs FP32 or FP64 storage of X, n > 0 and at most " +
                                        std::to_string(simt2_max_c()) + " free classes per chain");
    } else if (P.Km1 > maxct) {
      return fail(HMC_EUNSUPPORTED, "free classes per chain " + std::to_string(P.Km1) +
                                        " exceed the CUDA-core kernel's class bound " + std::to_string(maxct));
    } else if (!tc.S) {
      return fail(HMC_EUNSUPPORTED, "no CUDA-core tile configuration fits this problem (p too large for the cluster sizes "
                                    "available, or the requested tile does not fit)");
    } else {
      P.S = tc.S;
      P.BM = kSimtRows;
      P.CR = kSimtRows;
      P.NT = tc.NT;
      P.NWL = tc.NWL;
      P.NSTAGE = tc.NSTAGE;
      P.PC = tc.PC;
      P.smem = tc.smem;
      P.p_pad = P.S * P.PC;
      // A cluster's tiles run one after another through its pipeline (the
      // per-tile latency dominates small problems), and every cluster adds one
      // partial slice to the reduction: clusters beyond one per S SMs are
      // launched while each still gets about four tiles, or, up to one tile per
      // cluster, while the slices' bytes stay below X's (at least 8 MiB).
      const double slice = double(P.ct_launch) * P.p_pad * state_bytes(h);
      const double budget = std::max(double(P.n) * P.p_pad * dtype_bytes(h->xt), 8.0 * 1024 * 1024);
      const int64_t useful = std::max<int64_t>(
          {int64_t(nsm / P.S), (P.ntiles + 3) / 4, std::min<int64_t>(P.ntiles, int64_t(budget / slice))});
      P.nclusters = int(std::max<int64_t>(1, std::min<int64_t>({int64_t(tc.maxclu), P.ntiles, useful})));
    }
  }

  // X: convert on the device into the storage type, zero-padded columns.
  const size_t in_bytes = size_t(P.n) * P.p * (x_dtype == HMC_F64 ? 8 : 4);
  const void* Xd = X;
  void* tmp = nullptr;
  if (P.n > 0 && !is_device_ptr(X)) {
    HMC_CUDA(cudaMalloc(&tmp, in_bytes));
    HMC_CUDA(cudaMemcpyAsync(tmp, X, in_bytes, cudaMemcpyHostToDevice, h->stream));
    Xd = tmp;
  }
  const bool tiled = P.engine == 2 || P.engine == 3;   // X in 128-row tensor-core tiles
  const int64_t n_alloc = tiled ? (P.n + 127) / 128 * 128 : P.n;
  HMC_CUDA(cudaMalloc(&P.X, std::max<size_t>(16, size_t(n_alloc) * P.p_pad * xb)));
  if (h->xt == HMC_FP8E4M3) {
    HMC_CUDA(cudaMalloc(&P.xscale, size_t(P.p_pad) * sizeof(float)));
    HMC_CUDA(launch_fp8_scales(x_dtype, Xd, P.xscale, P.n, P.p, P.p_pad, h->stream));
  }
  if (P.n > 0) {
    if ((P.engine == 2 || P.engine == 3) && h->xt == HMC_FP8E4M3)
      HMC_CUDA(tc_x_to_tiles_fp8(x_dtype, Xd, P.xscale, P.X, P.n, P.p, P.p_pad, h->err_d, h->stream));
    else if (tiled)
      HMC_CUDA(tc_x_to_tiles(x_dtype, Xd, P.X, P.n, P.p, P.p_pad, h->err_d, h->stream));
    else
      HMC_CUDA(launch_convert_x(x_dtype, Xd, h->xt, P.X, P.xscale, P.n, P.p, P.p_pad, h->err_d, h->stream));
  }
  HMC_CUDA(cudaMalloc(&P.y, std::max<size_t>(16, size_t(P.n) * sizeof(int32_t))));
  if (P.n > 0)
    HMC_CUDA(cudaMemcpyAsync(P.y, y, size_t(P.n) * sizeof(int32_t), cudaMemcpyDefault, h->stream));
  HMC_CUDA(launch_check_labels(P.y, P.n, P.K, h->err_d, h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  if (tmp) cudaFree(tmp);
  HMC_TRY(check_device_error(h));

  // Partials, chain state and scalars.
  const size_t sb = state_bytes(h);
  P.state_elems = int64_t(h->max_chains) * P.Km1 * P.p_pad;
  HMC_CUDA(cudaMalloc(&P.gpart, size_t(P.nclusters) * P.state_elems * sb));
  P.nlparts = P.engine == 2 ? P.nclusters * P.S : P.engine == 3 ? P.tp2.gridA : P.engine == 4 ? int(simt2_ll_blocks(P.n)) : P.nclusters;
  HMC_CUDA(cudaMalloc(&P.lpart, size_t(P.nlparts) * h->max_chains * sizeof(double)));
  if (P.engine == 3) {
    const Tc2Plan& t2 = P.tp2;
    const int64_t ngroups = (h->max_chains + t2.gc - 1) / t2.gc;
    const size_t bbytes = size_t(ngroups) * (t2.p_pad / 64) * 2 * t2.N * 128;
    HMC_CUDA(cudaMalloc(&P.bbf, bbytes));
    HMC_CUDA(cudaMemsetAsync(P.bbf, 0, bbytes, h->stream));
    HMC_CUDA(cudaMalloc(&P.rbuf, size_t(P.ntiles) * ngroups * t2.NB * 16384));
    HMC_CUDA(cudaMalloc(&P.spart, size_t(t2.gridA) * t2.U * t2.N * 128 * sizeof(float)));
    HMC_CUDA(cudaMalloc(&P.sflag, size_t(t2.gridA) * sizeof(int)));
    HMC_CUDA(cudaMemsetAsync(P.sflag, 0, size_t(t2.gridA) * sizeof(int), h->stream));
  }
  if (P.engine == 4) {   // residuals and split logits of one chain group: [n][group_chains * Km1]
    HMC_CUDA(cudaMalloc(&P.rbuf, size_t(P.n) * P.ct_launch * sb));
    HMC_CUDA(cudaMalloc(&P.spart, size_t(P.fs) * P.n * P.ct_launch * sb));
  }
  if (P.engine == 2) {
    const TcPlan& tp = P.tp;
    HMC_CUDA(cudaMalloc(&P.bbf, size_t(2 * tp.N) * P.p_pad * 2));     // hi and lo terms
    HMC_CUDA(cudaMemsetAsync(P.bbf, 0, size_t(2 * tp.N) * P.p_pad * 2, h->stream));
  }
  for (StateSet* s : {&P.cs, &P.us}) {
    for (void** q : {&s->beta, &s->eta, &s->grad, &s->beta0, &s->grad0}) {
      HMC_CUDA(cudaMalloc(q, size_t(P.state_elems) * sb));
      HMC_CUDA(cudaMemsetAsync(*q, 0, size_t(P.state_elems) * sb, h->stream));
    }
  }
  {
    int dev = 0, nsm = 0;
    HMC_CUDA(cudaGetDevice(&dev));
    HMC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    P.glanes = update_group_lanes(int64_t(P.Km1) * P.p_pad, h->max_chains, P.nclusters, nsm);
  }
  P.nblk = update_blocks_per_chain(int64_t(P.Km1) * P.p_pad * P.glanes);
  HMC_CUDA(cudaMalloc(&P.logk, 2 * h->max_chains * sizeof(double)));
  HMC_CUDA(cudaMalloc(&P.logk0, h->max_chains * sizeof(double)));
  HMC_CUDA(cudaMalloc(&P.h0, h->max_chains * sizeof(double)));
  HMC_CUDA(cudaMalloc(&P.scal, size_t(h->max_chains) * P.nblk * 2 * sizeof(double)));
  HMC_CUDA(cudaMalloc(&P.tickets, (h->max_chains + 1) * sizeof(unsigned int)));
  HMC_CUDA(cudaMemsetAsync(P.tickets, 0, (h->max_chains + 1) * sizeof(unsigned int), h->stream));
  HMC_CUDA(cudaMalloc(&P.accept, h->max_chains * sizeof(int)));
  HMC_CUDA(cudaMalloc(&P.stats, h->max_chains * sizeof(hmc_chain_stats)));
  HMC_CUDA(cudaMalloc(&P.iter, 3 * sizeof(int64_t)));
  HMC_CUDA(cudaMemsetAsync(P.iter, 0, 3 * sizeof(int64_t), h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  return HMC_OK;
}

void free_problem(Problem& P) {
  void* ptrs[] = {P.X, P.y, P.xscale, P.gpart, P.lpart, P.cs.beta, P.cs.eta, P.cs.grad, P.cs.beta0, P.cs.grad0,
                  P.us.beta, P.us.eta, P.us.grad, P.us.beta0, P.us.grad0, P.logk, P.logk0, P.h0, P.scal,
                  P.tickets, P.accept, P.stats, P.iter, P.bbf, P.rbuf, P.spart, P.sflag};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

// ----------------------------------------------------------------- launches
hmc_status timer_pair(hmc_ctx* h, cudaEvent_t* a, cudaEvent_t* b, cudaEvent_t* m = nullptr) {
  FusedTimer& T = h->timer;
  while (T.ev.size() < 2 * (T.used + 1)) {
    cudaEvent_t e;
    HMC_CUDA(cudaEventCreate(&e));
    T.ev.push_back(e);
  }
  while (T.mid.size() < T.used + 1) {
    cudaEvent_t e;
    HMC_CUDA(cudaEventCreate(&e));
    T.mid.push_back(e);
    T.has_mid.push_back(0);
  }
  *a = T.ev[2 * T.used];
  *b = T.ev[2 * T.used + 1];
  T.has_mid[T.used] = m ? 1 : 0;
  if (m) *m = T.mid[T.used];
  T.used += 1;
  return HMC_OK;
}

// Harvest (synchronously) the fused-kernel durations recorded since the last harvest.
hmc_status timer_harvest(hmc_ctx* h) {
  FusedTimer& T = h->timer;
  if (T.used == 0) return HMC_OK;
  HMC_CUDA(cudaEventSynchronize(T.ev[2 * T.used - 1]));
  for (size_t i = 0; i < T.used; ++i) {
    float ms = 0.f;
    HMC_CUDA(cudaEventElapsedTime(&ms, T.ev[2 * i], T.ev[2 * i + 1]));
    h->timing_ms += ms;
    h->timing_launches += 1;
    if (T.has_mid[i]) {
      HMC_CUDA(cudaEventElapsedTime(&ms, T.ev[2 * i], T.mid[i]));
      h->timing_first_ms += ms;
    }
  }
  T.used = 0;
  return HMC_OK;
}

hmc_status run_lpg(hmc_ctx* h, Problem& P, StateSet& S, int chains, cudaStream_t stream) {
  if (P.n == 0) return HMC_OK;
  const size_t sb = state_bytes(h);
  if (P.engine == 3) {
    // Both passes for every chain of the call (the chain groups are inside the launches).
    const Tc2Plan& t2 = P.tp2;
    const int ngroups = (chains + t2.gc - 1) / t2.gc;
    HMC_CUDA(tc2_beta_boxes(static_cast<const float*>(S.beta), P.xscale, P.bbf, P.Km1, t2.gc, chains, t2.N, t2.p_pad, ngroups,
                            stream));
    const bool inject = h->inject_timeout;
    h->inject_timeout = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr, em = nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool timed = h->timing && (h->timing_seq++ % h->timing_period) == 0;
    if (timed) {
      HMC_CUDA(cudaStreamIsCapturing(stream, &cap));
      HMC_TRY(timer_pair(h, &e0, &e1, &em));
      HMC_CUDA(cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e0, stream, cudaEventRecordExternal)
                                                    : cudaEventRecord(e0, stream));
    }
    Tc2Launch L{};
    L.xs = P.X;
    L.xscale = P.xscale;
    L.fp8 = h->xt == HMC_FP8E4M3 ? 1 : 0;
    L.bs = P.bbf;
    L.y = P.y;
    L.rbuf = P.rbuf;
    L.spart = P.spart;
    L.sflag = P.sflag;
    L.lpart = P.lpart;
    L.lpart_cstride = h->max_chains;
    L.gpart = P.gpart;
    L.gpart_cstride = P.state_elems;
    L.err = h->err_d;
    L.n = P.n;
    L.Km1 = P.Km1;
    L.zlogit = P.zlogit;
    L.chains = chains;
    L.spin_limit = inject ? 0 : h->spin_limit;   // fault injection: every bounded wait gives up at once
    const cudaError_t le =
        tc2_launch(t2, L, stream, timed ? em : nullptr, cap == cudaStreamCaptureStatusActive);
    if (le != cudaSuccess) return fail(HMC_ECUDA, std::string("two-pass launch failed: ") + cudaGetErrorString(le));
    if (timed)
      HMC_CUDA(cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e1, stream, cudaEventRecordExternal)
                                                    : cudaEventRecord(e1, stream));
    return HMC_OK;
  }
  for (int c0 = 0; c0 < chains; c0 += P.group_chains) {
    const int c1 = std::min(chains, c0 + P.group_chains);
    const int C = (c1 - c0) * P.Km1;
    const void* beta = static_cast<const char*>(S.beta) + size_t(c0) * P.Km1 * P.p_pad * sb;
    void* gpart = static_cast<char*>(P.gpart) + size_t(c0) * P.Km1 * P.p_pad * sb;
    const bool inject = h->inject_timeout;
    h->inject_timeout = false;
    if (P.engine == 2)
      HMC_CUDA(tc_beta_to_tiles(static_cast<const float*>(beta), P.xscale, P.bbf, C, P.tp.N, P.p_pad, stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr, em = nullptr;
    // Inside a stream capture the events must become graph nodes.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool timed = h->timing && (h->timing_seq++ % h->timing_period) == 0;
    if (timed) {
      HMC_CUDA(cudaStreamIsCapturing(stream, &cap));
      HMC_TRY(timer_pair(h, &e0, &e1, P.engine == 4 ? &em : nullptr));
      HMC_CUDA(cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e0, stream, cudaEventRecordExternal)
                                                    : cudaEventRecord(e0, stream));
    }
    cudaError_t le;
    if (P.engine == 4) {
      Simt2Launch L{};
      L.X = P.X;
      L.y = P.y;
      L.beta = beta;
      L.rbuf = P.rbuf;
      L.zpart = P.spart;
      L.lrow = P.lpart + c0;
      L.lrow_stride = h->max_chains;
      L.gpart = gpart;
      L.gpart_cstride = P.state_elems;
      L.err = h->err_d;
      L.n = P.n;
      L.p_pad = P.p_pad;
      L.C = C;
      L.Km1 = P.Km1;
      L.chains = c1 - c0;
      L.zlogit = P.zlogit;
      L.Q = P.nclusters;
      L.FS = P.fs;
      le = simt2_launch(h->xt, L, stream, timed ? em : nullptr, cap == cudaStreamCaptureStatusActive);
    } else if (P.engine == 2) {
      TcLaunch L{};
      L.xs = P.X;
      L.xscale = P.xscale;
      L.fp8 = h->xt == HMC_FP8E4M3 ? 1 : 0;
      L.bs = P.bbf;
      L.n = P.n;
      L.p_pad = P.p_pad;
      L.C = C;
      L.Km1 = P.Km1;
      L.chains = c1 - c0;
      L.NST = P.NSTAGE;
      L.nclusters = P.nclusters;
      L.gpart = gpart;
      L.gpart_cstride = P.state_elems;
      L.lpart = P.lpart + c0;
      L.lpart_cstride = h->max_chains;
      L.y = P.y;
      L.err = h->err_d;
      L.spin_limit = h->spin_limit;
      L.inject_timeout = inject ? 1 : 0;
      L.zlogit = P.zlogit;
      le = tc_launch(P.tp, L, P.smem, stream);
    } else {
      LpgArgs a{};
      a.X = P.X;
      a.y = P.y;
      a.xscale = P.xscale;
      a.beta = beta;
      a.gpart = gpart;
      a.gpart_cstride = P.state_elems;
      a.lpart = P.lpart + c0;
      a.lpart_cstride = h->max_chains;
      a.err = h->err_d;
      a.n = P.n;
      a.p_pad = P.p_pad;
      a.PC = P.PC;
      a.C = C;
      a.Km1 = P.Km1;
      a.zlogit = P.zlogit;
      a.chains = c1 - c0;
      a.BM = P.BM;
      a.CR = P.CR;
      a.S = P.S;
      a.NT = P.NT;
      a.NWL = P.NWL;
      a.NSTAGE = P.NSTAGE;
      a.nclusters = P.nclusters;
      a.ntiles = P.ntiles;
      a.spin_limit = h->spin_limit;
      a.inject_timeout = inject ? 1 : 0;
      le = simt_launch(h->xt, h->st, a, P.smem, stream, P.ct_launch);
    }
    if (le != cudaSuccess) {
      char buf[256];
      std::snprintf(buf, sizeof(buf), "fused launch failed (%s): engine=%d clusters=%d x S=%d, smem=%zu, C=%d, BM=%d, NSTAGE=%d",
                    cudaGetErrorString(le), P.engine, P.nclusters, P.S, P.smem, C, P.BM, P.NSTAGE);
      return fail(HMC_ECUDA, buf);
    }
    if (timed)
      HMC_CUDA(cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e1, stream, cudaEventRecordExternal)
                                                    : cudaEventRecord(e1, stream));
  }
  return HMC_OK;
}

LpgArgs batched_args(hmc_ctx* h, Problem& P, StateSet& S) {
  LpgArgs a{};
  a.X = P.X;
  a.y = P.y;
  a.xscale = P.xscale;
  a.beta = S.beta;
  a.gpart = P.gpart;
  a.gpart_cstride = P.state_elems;
  a.lpart = P.lpart;
  a.lpart_cstride = h->max_chains;
  a.err = h->err_d;
  a.n = P.n;
  a.p_pad = P.p_pad;
  a.PC = P.PC;
  a.C = h->max_chains * P.Km1;
  a.Km1 = P.Km1;
  a.zlogit = P.zlogit;
  a.chains = h->max_chains;
  a.BM = P.BM;
  a.CR = P.CR;
  a.S = h->b_S;
  a.NT = h->b_NT;
  a.NWL = h->b_NWL;
  a.NSTAGE = P.NSTAGE;
  a.nclusters = P.nclusters;
  a.ntiles = P.ntiles;
  a.spin_limit = h->spin_limit;
  a.inject_timeout = 0;
  return a;
}

// Decide whether every problem of a batch handle can share one fused launch,
// and if so build the device tables and the cluster split (by work).
hmc_status setup_batched(hmc_ctx* h) {
  const int m = int(h->probs.size());
  if (m < 2) return HMC_OK;
  int NWC = 1, C = 1, S = h->probs[0].S;
  for (Problem& P : h->probs) {
    if (P.engine != 1 || P.n == 0 || P.group_chains < h->max_chains || P.S != S) return HMC_OK;
    NWC = std::max(NWC, (P.PC + 127) / 128);
    C = std::max(C, P.ct_launch);
  }
  if (NWC > simt_max_grad_warps(h->xt, C)) return HMC_OK;
  const int NWL = simt_logit_warps(NWC);
  const int NT = 32 * (NWC + NWL + 1);
  int dev = 0, smem_max = 0;
  HMC_CUDA(cudaGetDevice(&dev));
  HMC_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  size_t smem = 0;
  for (Problem& P : h->probs)
    smem = std::max(smem, simt_smem_bytes(h->xt, h->st, C, P.PC, S, NWL, P.NSTAGE));
  if (smem + 1024 > size_t(smem_max)) return HMC_OK;
  HMC_CUDA(simt_prepare_batched(h->xt, C, S));
  int cap = 0;
  HMC_CUDA(simt_max_active_clusters_batched(h->xt, C, smem, S, NT, &cap));
  if (cap < 1) return HMC_OK;
  double total = 0.0;
  for (Problem& P : h->probs) total += double(P.ntiles) * P.BM * P.PC;
  std::vector<int> first(m + 1, 0);
  for (int b = 0; b < m; ++b) {
    Problem& P = h->probs[b];
    const double share = double(P.ntiles) * P.BM * P.PC / total;
    int nc = int(std::lround(share * cap));
    nc = std::max(1, std::min(nc, P.nclusters));
    P.nclusters = nc;
    P.nlparts = nc;
    first[b + 1] = first[b] + nc;
  }
  h->b_S = S;
  h->b_NT = NT;
  h->b_NWL = NWL;
  h->b_CT = C;
  h->b_smem = smem;
  h->b_total_clusters = first[m];
  std::vector<LpgArgs> table(2 * m);
  for (int b = 0; b < m; ++b) {
    table[b] = batched_args(h, h->probs[b], h->probs[b].cs);
    table[m + b] = batched_args(h, h->probs[b], h->probs[b].us);
  }
  HMC_CUDA(cudaMalloc(&h->b_table, table.size() * sizeof(LpgArgs)));
  HMC_CUDA(cudaMalloc(&h->b_first, first.size() * sizeof(int)));
  HMC_CUDA(cudaMemcpy(h->b_table, table.data(), table.size() * sizeof(LpgArgs), cudaMemcpyHostToDevice));
  HMC_CUDA(cudaMemcpy(h->b_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice));
  h->batched = true;
  return HMC_OK;
}

// Tensor-core engine: one launch for every problem when they share the
// cluster size and each runs all chains in one group.  Clusters are split by
// work (n p); the dynamic shared memory is the largest any problem needs.
hmc_status setup_batched_tc(hmc_ctx* h) {
  const int m = int(h->probs.size());
  if (m < 2) return HMC_OK;
  const int S = h->probs[0].S;
  for (Problem& P : h->probs)
    if (P.engine != 2 || P.n == 0 || P.group_chains < h->max_chains || P.S != S) return HMC_OK;
  int dev = 0, smem_max = 0;
  HMC_CUDA(cudaGetDevice(&dev));
  HMC_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const bool fp8 = h->xt == HMC_FP8E4M3;
  // The batched kernel keeps the problem's arguments in static shared memory:
  // leave room for them by taking ring slots off problems that need it.
  const size_t limit = size_t(smem_max) - 512;
  size_t smem = 0;
  for (Problem& P : h->probs) {
    while (P.smem > limit && P.NSTAGE > 2) {
      P.NSTAGE -= 1;
      P.smem = std::max(tc_smem_bytes(P.tp, P.NSTAGE, h->max_chains, fp8), size_t(116 * 1024));
    }
    if (P.smem > limit) return HMC_OK;
    smem = std::max(smem, P.smem);
  }
  HMC_CUDA(tc_prepare_batched(smem, S, fp8));
  int cap = 0;
  if (tc_max_active_clusters_batched(smem, S, fp8, &cap) != cudaSuccess) {
    cudaGetLastError();
    return HMC_OK;
  }
  if (cap < 1) return HMC_OK;
  double total = 0.0;
  for (Problem& P : h->probs) total += double(P.n) * P.p_pad;
  std::vector<int> first(m + 1, 0);
  std::vector<TcPlan> plans(m);
  std::vector<TcLaunch> launches(m);
  std::vector<TcBetaBox> boxes(2 * m);
  int64_t max_elems = 1;
  for (int b = 0; b < m; ++b) {
    Problem& P = h->probs[b];
    int nc = int(std::lround(double(P.n) * P.p_pad / total * cap));
    nc = std::max(1, std::min(nc, P.nclusters));   // partial buffers hold P.nclusters
    P.nclusters = nc;
    P.nlparts = nc * S;
    first[b + 1] = first[b] + nc;
    plans[b] = P.tp;
    TcLaunch& L = launches[b];
    L = TcLaunch{};
    L.xs = P.X;
    L.xscale = P.xscale;
    L.fp8 = fp8 ? 1 : 0;
    L.bs = P.bbf;
    L.n = P.n;
    L.p_pad = P.p_pad;
    L.C = h->max_chains * P.Km1;
    L.Km1 = P.Km1;
    L.chains = h->max_chains;
    L.NST = P.NSTAGE;
    L.nclusters = nc;
    L.gpart = P.gpart;
    L.gpart_cstride = P.state_elems;
    L.lpart = P.lpart;
    L.lpart_cstride = h->max_chains;
    L.y = P.y;
    L.err = h->err_d;
    L.spin_limit = h->spin_limit;
    L.inject_timeout = 0;
    L.zlogit = P.zlogit;
    for (int w = 0; w < 2; ++w)
      boxes[w * m + b] = TcBetaBox{static_cast<const float*>(w == 0 ? P.cs.beta : P.us.beta), P.xscale, P.bbf, P.Km1,
                                   P.tp.N, P.p_pad};
    max_elems = std::max<int64_t>(max_elems, int64_t(P.tp.N) * P.p_pad);
  }
  HMC_CUDA(tc_upload_batch(plans.data(), launches.data(), m, &h->tb_table));
  HMC_CUDA(tc_upload_beta_table(boxes.data(), 2 * m, &h->tb_beta));
  HMC_CUDA(cudaMalloc(&h->b_first, first.size() * sizeof(int)));
  HMC_CUDA(cudaMemcpy(h->b_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice));
  h->b_S = S;
  h->b_smem = smem;
  h->b_total_clusters = first[m];
  h->tb_max_elems = max_elems;
  h->tc_batched = true;
  return HMC_OK;
}

// The fused pass for every problem: one launch for a batched handle, else one
// launch per problem (and per chain group).
hmc_status run_lpg_all(hmc_ctx* h, bool chain_state, int chains, cudaStream_t stream) {
  if (!h->batched && !h->tc_batched) {
    for (Problem& P : h->probs) HMC_TRY(run_lpg(h, P, chain_state ? P.cs : P.us, chains, stream));
    return HMC_OK;
  }
  const int mtc = int(h->probs.size());
  if (h->tc_batched)   // operand boxes of every problem's coefficients (one launch, not timed)
    HMC_CUDA(tc_beta_to_tiles_batched(static_cast<const char*>(h->tb_beta) + (chain_state ? 0 : 1) * mtc *
                                          size_t(tc_beta_job_bytes()),
                                      mtc, chains, h->tb_max_elems, stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool timed = h->timing && (h->timing_seq++ % h->timing_period) == 0;
  if (timed) {
    HMC_CUDA(cudaStreamIsCapturing(stream, &cap));
    HMC_TRY(timer_pair(h, &e0, &e1));
    HMC_CUDA(cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e0, stream, cudaEventRecordExternal)
                                                  : cudaEventRecord(e0, stream));
  }
  const int m = int(h->probs.size());
  const cudaError_t le =
      h->tc_batched
          ? tc_launch_batched(h->tb_table, h->b_first, m, chains, h->b_total_clusters, h->b_S,
                              h->xt == HMC_FP8E4M3, h->b_smem, stream)
          : simt_launch_batched(h->xt, h->b_CT, h->b_table + (chain_state ? 0 : m), h->b_first, m, chains,
                                h->b_total_clusters, h->b_S, h->b_NT, h->b_smem, stream);
  if (le != cudaSuccess) return fail(HMC_ECUDA, std::string("batched fused launch failed: ") + cudaGetErrorString(le));
  if (timed)
    HMC_CUDA(cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e1, stream, cudaEventRecordExternal)
                                                  : cudaEventRecord(e1, stream));
  return HMC_OK;
}

UpdateArgs make_update(hmc_ctx* h, Problem& P, StateSet& S, int which_logk, int chains, double eps, int b) {
  UpdateArgs u{};
  u.beta = S.beta;
  u.eta = S.eta;
  u.grad = S.grad;
  u.beta0 = S.beta0;
  u.grad0 = S.grad0;
  u.gpart = P.gpart;
  u.gpart_cstride = P.state_elems;
  u.nparts = P.n > 0 ? P.nclusters : 0;
  u.glanes = P.glanes;
  u.lpart = P.lpart;
  u.lpart_cstride = h->max_chains;
  u.nlparts = P.n > 0 ? P.nlparts : 0;
  u.logk = P.logk + which_logk * h->max_chains;
  u.logk0 = P.logk0;
  u.h0 = P.h0;
  u.scal = P.scal;
  u.tickets = P.tickets;
  u.accept = P.accept;
  u.stats = P.stats;
  u.temps = nullptr;
  u.iter = P.iter;
  u.local_iter = P.iter + 1;
  u.samples = nullptr;
  u.thin = 1;
  u.sample_slot_stride = 0;
  u.chains_word_hi = b;
  u.err = h->err_d;
  u.p = P.p;
  u.p_pad = P.p_pad;
  u.Km1 = P.Km1;
  u.ku = P.ku;
  u.chains = chains;
  u.nblk = P.nblk;
  u.prior_kind = h->prior_kind;
  u.prior_scale = h->prior_scale;
  u.eps = eps;
  u.seed = reinterpret_cast<const uint64_t*>(P.iter + 2);
  return u;
}

hmc_status validate_opts(const hmc_opts* o) {
  if (!o) return HMC_OK;
  if (o->x_storage < HMC_F64 || o->x_storage > HMC_FP8E4M3) return fail(HMC_EINVAL, "opts.x_storage out of range");
  if (o->state != HMC_F64 && o->state != HMC_F32) return fail(HMC_EINVAL, "opts.state must be HMC_F64 or HMC_F32");
  if ((o->x_storage == HMC_F64) != (o->state == HMC_F64))
    return fail(HMC_EINVAL, "HMC_F64 storage of X goes with HMC_F64 state, and only with it");
  if (o->max_chains < 1 || o->max_chains > 4096) return fail(HMC_EINVAL, "opts.max_chains must be in [1, 4096]");
  if (o->engine < 0 || o->engine > 4) return fail(HMC_EINVAL, "opts.engine must be 0, 1, 2, 3 or 4");
  if (o->spin_limit < 0) return fail(HMC_EINVAL, "opts.spin_limit must be >= 0");
  const int* t = o->tile;
  if (t[0] < 0 || t[0] > 16) return fail(HMC_EINVAL, "opts.tile[0] (cluster size) must be in [0, 16]");
  if (o->engine == 3 && (t[0] > 4 || t[1] || t[2] || t[3]))
    return fail(HMC_EINVAL, "on the two-pass engine only opts.tile[0] (row tiles per first-pass unit, 1..4) applies");
  if (o->engine == 4 && (t[0] || t[1] || t[2] || t[3]))
    return fail(HMC_EINVAL, "the two-pass CUDA-core engine takes no tile options");
  if (t[1] < 0 || t[1] > kTcMaxDepth)
    return fail(HMC_EINVAL, "opts.tile[1] (tensor-core exchange depth) must be in [0, " + std::to_string(kTcMaxDepth) + "]");
  if (t[2] < 0 || t[2] > kTcMaxDepth)
    return fail(HMC_EINVAL, "opts.tile[2] (tensor-core sweep lookahead) must be in [0, " + std::to_string(kTcMaxDepth) + "]");
  if (t[3] != 0 && (t[3] < 2 || t[3] > 6)) return fail(HMC_EINVAL, "opts.tile[3] (ring chunks) must be 0 or in [2, 6]");
  if (o->layout < HMC_LAYOUT_FREE || o->layout > HMC_LAYOUT_UNCONSTRAINED)
    return fail(HMC_EINVAL, "opts.layout must be HMC_LAYOUT_FREE, HMC_LAYOUT_MASKED or HMC_LAYOUT_UNCONSTRAINED");
  return HMC_OK;
}

void build_description(hmc_ctx* h) {
  const int e0 = h->probs.empty() ? 1 : h->probs[0].engine;
  std::string s = "{\"engine\": \"" + std::string(e0 == 1 ? "simt" : e0 == 2 ? "tcgen05" : e0 == 3 ? "tcgen05_2pass" : "simt_2pass") +
                  "\", \"batched_launch\": " + std::string(h->batched || h->tc_batched ? "true" : "false") +
                  ", \"layout\": " + std::to_string(h->layout) +
                  ", \"x_storage\": " + std::to_string(h->xt) +
                  ", \"state\": " + std::to_string(h->st) + ", \"max_chains\": " + std::to_string(h->max_chains) +
                  ", \"problems\": [";
  for (size_t b = 0; b < h->probs.size(); ++b) {
    const Problem& P = h->probs[b];
    char buf[512];
    std::snprintf(buf, sizeof(buf),
                  "%s{\"n\": %lld, \"p\": %d, \"K\": %d, \"p_pad\": %d, \"S\": %d, \"BM\": %d, \"CR\": %d, "
                  "\"NT\": %d, \"NSTAGE\": %d, \"PC\": %d, \"nclusters\": %d, \"smem\": %zu, \"group_chains\": %d, "
                  "\"ct\": %d, \"nz\": %d, \"depth\": %d, \"lookahead\": %d}",
                  b ? ", " : "", (long long)P.n, P.p, P.K, P.p_pad, P.S, P.BM, P.CR, P.NT, P.NSTAGE, P.PC, P.nclusters,
                  P.smem, P.group_chains, P.ct_launch, P.engine == 2 ? P.tp.nz : 0, P.engine == 2 ? P.tp.slots : 0,
                  P.engine == 2 ? P.tp.la : 0);
    s += buf;
    if (P.engine == 3) {
      const Tc2Plan& t = P.tp2;
      std::snprintf(buf, sizeof(buf),
                    ", \"pass_a\": {\"grid\": %d, \"tiles_per_unit\": %d, \"chain_group\": %d, \"N\": %d, \"ring\": %d, \"smem\": %zu}, "
                    "\"pass_b\": {\"feature_blocks\": %d, \"feature_groups\": %d, \"row_ranges\": %d, \"ring\": %d, "
                    "\"r_slots\": %d, \"smem\": %zu}",
                    t.gridA, t.U, t.gc, t.N, t.nstA, t.smemA, t.MB, t.nfg, t.Q, t.nstB, t.nrsB, t.smemB);
      s.insert(s.size() - 1, buf);   // inside this problem's object
    }
  }
  s += "]}";
  h->desc = s;
}

hmc_status create_common(int32_t nprob, const void* const* X, hmc_dtype x_dtype, const int32_t* const* y,
                         const int64_t* n, const int64_t* p, const int32_t* K, hmc_prior_kind prior,
                         double prior_scale, const hmc_opts* opts, hmc_handle* out) {
  g_last_error.clear();
  if (!out) return fail(HMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || nprob > 4096) return fail(HMC_EINVAL, "nprob must be in [1, 4096]");
  if (!X || !y || !n || !p || !K) return fail(HMC_EINVAL, "NULL array argument");
  if (x_dtype != HMC_F64 && x_dtype != HMC_F32) return fail(HMC_EINVAL, "x_dtype must be HMC_F64 or HMC_F32");
  if (prior != HMC_PRIOR_GAUSSIAN && prior != HMC_PRIOR_CAUCHY) return fail(HMC_EINVAL, "unknown prior kind");
  if (!(prior_scale > 0.0) || !std::isfinite(prior_scale)) return fail(HMC_EINVAL, "prior_scale must be finite and > 0");
  hmc_opts o;
  hmc_default_opts(&o);
  if (opts) o = *opts;
  HMC_TRY(validate_opts(&o));
  for (int b = 0; b < nprob; ++b) {
    if (n[b] < 0 || n[b] > (int64_t(1) << 40)) return fail(HMC_EINVAL, "n out of range");
    if (p[b] < 1 || p[b] > (int64_t(1) << 24)) return fail(HMC_EINVAL, "p out of range");
    if (K[b] < 2 || K[b] > 1024) return fail(HMC_EINVAL, "K must be in [2, 1024]");
    if (n[b] > 0 && (!X[b] || !y[b])) return fail(HMC_EINVAL, "NULL X or y with n > 0");
  }
  hmc_ctx* h = new hmc_ctx();
  h->xt = o.x_storage;
  h->st = o.state;
  h->prior_kind = prior;
  h->prior_scale = prior_scale;
  h->max_chains = o.max_chains;
  h->engine = o.engine;
  h->layout = o.layout;
  h->spin_limit = o.spin_limit > 0 ? o.spin_limit : (1ll << 22);
  h->stream = static_cast<cudaStream_t>(o.stream);
  for (int i = 0; i < 4; ++i) h->tile[i] = o.tile[i];
  if (const char* f = std::getenv("HMC_FAULT")) h->inject_timeout = std::strcmp(f, "timeout") == 0;
  auto cleanup = [&](hmc_status s) {
    hmc_destroy(h);
    return s;
  };
  if (cudaMalloc(&h->err_d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(HMC_ENOMEM, "cudaMalloc of the error word failed");
  }
  if (cudaMemsetAsync(h->err_d, 0, sizeof(int), h->stream) != cudaSuccess) return cleanup(fail(HMC_ECUDA, "memset"));
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cleanup(fail(HMC_ECUDA, "cudaStreamCreateWithFlags failed"));
  h->probs.resize(nprob);
  for (int b = 0; b < nprob; ++b) {
    Problem& P = h->probs[b];
    P.n = n[b];
    P.p = int32_t(p[b]);
    P.K = K[b];
    P.Km1 = (h->layout == HMC_LAYOUT_UNCONSTRAINED) ? K[b] : K[b] - 1;
    P.ku = (h->layout == HMC_LAYOUT_FREE) ? K[b] - 1 : K[b];
    P.zlogit = (h->layout == HMC_LAYOUT_UNCONSTRAINED) ? 0 : 1;
  }
  // A batch on the CUDA-core engine shares one cluster size (the largest any
  // problem needs) so that one fused launch can serve every problem.
  const bool want_batch =
      nprob > 1 && !((h->xt == HMC_BF16 || h->xt == HMC_FP8E4M3) && h->engine != 1) && !h->tile[0];
  // A batch on the tensor-core engine shares the smallest cluster size whose
  // tile plan fits every problem with all chains in one launch.
  bool want_tc_batch = nprob > 1 && (h->xt == HMC_BF16 || h->xt == HMC_FP8E4M3) && h->engine != 1 && !h->tile[0];
  if (want_tc_batch) {
    int S_tc = 0;
    for (int S : {1, 2, 4, 8, 16}) {
      bool ok = true;
      for (Problem& P : h->probs) {
        TcPlan pl;
        if (P.n == 0 || !tc_plan(P.p, h->max_chains * P.Km1, S, &pl)) {
          ok = false;
          break;
        }
      }
      if (ok) {
        S_tc = S;
        break;
      }
    }
    if (S_tc)
      h->tile[0] = S_tc;
    else
      want_tc_batch = false;
  }
  if (want_batch) {
    // Smallest cluster whose column slices fit the block for every problem.
    int S = 1;
    for (Problem& P : h->probs) {
      const int maxct = simt_max_ct(h->xt);
      const int g = std::max(1, std::min(h->max_chains, maxct / std::max(1, P.Km1)));
      const int64_t cols = int64_t(128) * simt_max_grad_warps(h->xt, std::min(maxct, g * P.Km1));
      while (S < 16 && (int64_t(P.p) + S - 1) / S > cols) S *= 2;
    }
    h->tile[0] = S;
  }
  for (int b = 0; b < nprob; ++b) {
    Problem& P = h->probs[b];
    hmc_status s = setup_problem(h, P, X[b], x_dtype, y[b]);
    if (s != HMC_OK) return cleanup(s);
    h->chain_size += int64_t(P.ku) * P.p;
  }
  if (want_batch) {
    h->tile[0] = 0;
    hmc_status s = setup_batched(h);
    if (s != HMC_OK) return cleanup(s);
  }
  if (want_tc_batch) {
    h->tile[0] = 0;
    hmc_status s = setup_batched_tc(h);
    if (s != HMC_OK) return cleanup(s);
  }
  build_description(h);
  *out = h;
  return HMC_OK;
}

int64_t block_offset(const hmc_ctx* h, int b, int chains) {
  int64_t off = 0;
  for (int q = 0; q < b; ++q) off += int64_t(chains) * h->probs[q].ku * h->probs[q].p;
  return off;
}

// Pack a user beta-layout buffer (device) into the padded state of each problem.
hmc_status pack_all(hmc_ctx* h, const void* user_dev, int chains, bool chain_state, void* StateSet::*field) {
  const size_t sb = state_bytes(h);
  for (size_t b = 0; b < h->probs.size(); ++b) {
    Problem& P = h->probs[b];
    StateSet& S = chain_state ? P.cs : P.us;
    const char* src = static_cast<const char*>(user_dev) + size_t(block_offset(h, int(b), chains)) * sb;
    HMC_CUDA(launch_pack(h->st, src, S.*field, chains, P.ku, P.Km1, P.p, P.p_pad, h->stream));
  }
  return HMC_OK;
}

hmc_status unpack_all(hmc_ctx* h, void* user_dev, int chains, bool chain_state, void* StateSet::*field) {
  const size_t sb = state_bytes(h);
  for (size_t b = 0; b < h->probs.size(); ++b) {
    Problem& P = h->probs[b];
    StateSet& S = chain_state ? P.cs : P.us;
    char* dst = static_cast<char*>(user_dev) + size_t(block_offset(h, int(b), chains)) * sb;
    HMC_CUDA(launch_unpack(h->st, S.*field, dst, chains, P.ku, P.Km1, P.p, P.p_pad, h->stream));
  }
  return HMC_OK;
}

hmc_status copy_logk(hmc_ctx* h, double* user_dev, int chains, int which) {
  for (size_t b = 0; b < h->probs.size(); ++b)
    HMC_CUDA(cudaMemcpyAsync(user_dev + b * chains, h->probs[b].logk + which * h->max_chains,
                             size_t(chains) * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return HMC_OK;
}

hmc_status check_chains(hmc_ctx* h, int chains) {
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (chains < 1 || chains > h->max_chains)
    return fail(HMC_EINVAL, "chains must be in [1, max_chains=" + std::to_string(h->max_chains) + "]");
  return HMC_OK;
}

// log K and gradient at the state in `S` for every problem.
// Enqueue `body` (work on h->stream) directly, or through the call graph of
// `slot` when `cacheable` (device buffers only, no timing events, no pending
// fault injection): the second identical call in a row is captured on the
// private stream and launched as a graph, later ones replay it.
template <typename F>
hmc_status run_cached(hmc_ctx* h, int slot, std::vector<uint64_t> key, bool cacheable, F body) {
  hmc_ctx::CallGraph& g = h->cg[slot];
  key.push_back(uint64_t(reinterpret_cast<uintptr_t>(h->stream)));
  if (!cacheable) {
    g.seen = false;
    return body();
  }
  if (g.exec && g.key == key) {
    HMC_CUDA(cudaGraphLaunch(g.exec, h->stream));
    return HMC_OK;
  }
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!g.seen || g.key != key) {
    g.key = key;
    g.seen = true;
    return body();
  }
  cudaStream_t user = h->stream;
  HMC_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  h->stream = h->cap_stream;
  const hmc_status st = body();
  h->stream = user;
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
  if (st == HMC_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st != HMC_OK) {
    g.exec = nullptr;
    g.seen = false;
    return st;
  }
  if (ce != cudaSuccess) {
    g.exec = nullptr;
    g.seen = false;
    return fail(HMC_ECUDA, std::string("call graph capture failed: ") + cudaGetErrorString(ce));
  }
  HMC_CUDA(cudaGraphLaunch(g.exec, h->stream));
  return HMC_OK;
}

uint64_t key_of(const void* p) { return uint64_t(reinterpret_cast<uintptr_t>(p)); }

// Gradient and log K of the chains' (or the user scratch's) coefficients; the
// reduction also writes them to `ugrad` (user beta layout) and `ulogk`
// ([problem][chains]) when given.
hmc_status eval_state(hmc_ctx* h, bool chain_state, int chains, void* ugrad = nullptr, double* ulogk = nullptr) {
  HMC_TRY(run_lpg_all(h, chain_state, chains, h->stream));
  const size_t sb = state_bytes(h);
  for (size_t b = 0; b < h->probs.size(); ++b) {
    Problem& P = h->probs[b];
    StateSet& S = chain_state ? P.cs : P.us;
    UpdateArgs u = make_update(h, P, S, chain_state ? 0 : 1, chains, 0.0, int(b));
    if (ugrad) u.ugrad = static_cast<char*>(ugrad) + size_t(block_offset(h, int(b), chains)) * sb;
    if (ulogk) u.ulogk = ulogk + b * chains;
    HMC_CUDA(launch_reduce_update(h->st, u, UPD_SCALARS, h->stream));
  }
  return HMC_OK;
}

}  // namespace

namespace hmc {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace hmc

// =================================================================== C ABI
extern "C" {

void hmc_default_opts(hmc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->x_storage = HMC_F32;
  o->state = HMC_F32;
  o->max_chains = 1;
  o->engine = 0;
  o->spin_limit = 0;
  o->stream = nullptr;
}

const char* hmc_version(void) { return "libhmc 0.1 (sm_103a)"; }

const char* hmc_last_error(void) { return g_last_error.c_str(); }

hmc_status hmc_create(const void* X, hmc_dtype x_dtype, const int32_t* y, int64_t n, int64_t p, int32_t K,
                      hmc_prior_kind prior, double prior_scale, const hmc_opts* opts, hmc_handle* out) {
  const void* Xs[1] = {X};
  const int32_t* ys[1] = {y};
  return create_common(1, Xs, x_dtype, ys, &n, &p, &K, prior, prior_scale, opts, out);
}

hmc_status hmc_create_batch(int32_t nprob, const void* const* X, hmc_dtype x_dtype, const int32_t* const* y,
                            const int64_t* n, const int64_t* p, const int32_t* K, hmc_prior_kind prior,
                            double prior_scale, const hmc_opts* opts, hmc_handle* out) {
  return create_common(nprob, X, x_dtype, y, n, p, K, prior, prior_scale, opts, out);
}

hmc_status hmc_destroy(hmc_handle h) {
  if (!h) return HMC_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (Problem& P : h->probs) free_problem(P);
  if (h->err_d) cudaFree(h->err_d);
  if (h->temps_d) cudaFree(h->temps_d);
  for (void* s : h->staging)
    if (s) cudaFree(s);
  for (cudaEvent_t e : h->timer.ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->timer.mid) cudaEventDestroy(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (auto& g : h->cg)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->b_table) cudaFree(h->b_table);
  if (h->b_first) cudaFree(h->b_first);
  if (h->tb_table) cudaFree(h->tb_table);
  if (h->tb_beta) cudaFree(h->tb_beta);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return HMC_OK;
}

int64_t hmc_chain_size(hmc_handle h) { return h ? h->chain_size : -1; }

hmc_status hmc_logpost_grad(hmc_handle h, const void* beta, int32_t chains, double* logpost, void* grad) {
  g_last_error.clear();
  HMC_TRY(check_chains(h, chains));
  if (!beta) return fail(HMC_EINVAL, "beta is NULL");
  const size_t bytes = size_t(chains) * h->chain_size * state_bytes(h);
  const void* bd = nullptr;
  HMC_TRY(dev_in(h, 0, beta, bytes, &bd));
  bool gh = false, lh = false;
  void* gd = nullptr;
  void* ld = nullptr;
  HMC_TRY(dev_out(h, 1, grad, bytes, &gd, &gh));
  HMC_TRY(dev_out(h, 2, logpost, h->probs.size() * chains * sizeof(double), &ld, &lh));
  const bool cacheable = bd == beta && !gh && !lh && !h->timing && !h->inject_timeout;
  HMC_TRY(run_cached(h, 0, {uint64_t(chains), key_of(bd), key_of(gd), key_of(ld)}, cacheable, [&]() -> hmc_status {
    HMC_TRY(pack_all(h, bd, chains, false, &StateSet::beta));
    return eval_state(h, false, chains, gd, static_cast<double*>(ld));
  }));
  if (gh) HMC_CUDA(cudaMemcpyAsync(grad, gd, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (lh)
    HMC_CUDA(cudaMemcpyAsync(logpost, ld, h->probs.size() * chains * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (gh || lh || beta != bd || h->timing) {
    HMC_TRY(check_device_error(h));
    if (h->timing) HMC_TRY(timer_harvest(h));
  }
  return HMC_OK;
}

hmc_status hmc_leapfrog(hmc_handle h, void* beta, void* eta, void* grad, double* logpost, int32_t chains, int32_t L,
                        double eps) {
  g_last_error.clear();
  HMC_TRY(check_chains(h, chains));
  if (!beta || !eta) return fail(HMC_EINVAL, "beta and eta must not be NULL");
  if (L < 0) return fail(HMC_EINVAL, "L must be >= 0");
  if (!std::isfinite(eps)) return fail(HMC_EINVAL, "eps must be finite");
  const size_t bytes = size_t(chains) * h->chain_size * state_bytes(h);
  bool bh = false, eh = false, gh = false, lh = false;
  void *bd = nullptr, *ed = nullptr, *gd = nullptr, *ld = nullptr;
  HMC_TRY(dev_out(h, 0, beta, bytes, &bd, &bh));
  HMC_TRY(dev_out(h, 1, eta, bytes, &ed, &eh));
  HMC_TRY(dev_out(h, 2, grad, bytes, &gd, &gh));
  HMC_TRY(dev_out(h, 3, logpost, h->probs.size() * chains * sizeof(double), &ld, &lh));
  if (bh) HMC_CUDA(cudaMemcpyAsync(bd, beta, bytes, cudaMemcpyHostToDevice, h->stream));
  if (eh) HMC_CUDA(cudaMemcpyAsync(ed, eta, bytes, cudaMemcpyHostToDevice, h->stream));
  if (gh) HMC_CUDA(cudaMemcpyAsync(gd, grad, bytes, cudaMemcpyHostToDevice, h->stream));
  uint64_t eps_bits = 0;
  std::memcpy(&eps_bits, &eps, sizeof(eps_bits));
  const bool cacheable = !bh && !eh && !gh && !lh && !h->timing && !h->inject_timeout;
  HMC_TRY(run_cached(h, 1, {uint64_t(chains), uint64_t(L), eps_bits, key_of(bd), key_of(ed), key_of(gd), key_of(ld)},
                     cacheable, [&]() -> hmc_status {
    HMC_TRY(pack_all(h, bd, chains, false, &StateSet::beta));
    HMC_TRY(pack_all(h, ed, chains, false, &StateSet::eta));
    if (gd) {
      HMC_TRY(pack_all(h, gd, chains, false, &StateSet::grad));
    }
    if (!gd || L == 0) HMC_TRY(eval_state(h, false, chains));
    if (L > 0) {
      for (size_t b = 0; b < h->probs.size(); ++b) {
        UpdateArgs u = make_update(h, h->probs[b], h->probs[b].us, 1, chains, eps, int(b));
        HMC_CUDA(launch_leap_start(h->st, u, h->stream));
      }
      for (int l = 1; l <= L; ++l) {
        HMC_TRY(run_lpg_all(h, false, chains, h->stream));
        const int mode = (l < L) ? (UPD_ETA_FULL | UPD_BETA) : (UPD_ETA_HALF | UPD_SCALARS);
        for (size_t b = 0; b < h->probs.size(); ++b) {
          UpdateArgs u = make_update(h, h->probs[b], h->probs[b].us, 1, chains, eps, int(b));
          HMC_CUDA(launch_reduce_update(h->st, u, mode, h->stream));
        }
      }
    }
    HMC_TRY(unpack_all(h, bd, chains, false, &StateSet::beta));
    HMC_TRY(unpack_all(h, ed, chains, false, &StateSet::eta));
    if (gd) HMC_TRY(unpack_all(h, gd, chains, false, &StateSet::grad));
    if (ld) HMC_TRY(copy_logk(h, static_cast<double*>(ld), chains, 1));
    return HMC_OK;
  }));
  if (bh) HMC_CUDA(cudaMemcpyAsync(beta, bd, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (eh) HMC_CUDA(cudaMemcpyAsync(eta, ed, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (gh) HMC_CUDA(cudaMemcpyAsync(grad, gd, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (lh)
    HMC_CUDA(cudaMemcpyAsync(logpost, ld, h->probs.size() * chains * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (bh || eh || gh || lh || h->timing) {
    HMC_TRY(check_device_error(h));
    if (h->timing) HMC_TRY(timer_harvest(h));
  }
  return HMC_OK;
}

hmc_status hmc_sample_tempered(hmc_handle h, int32_t chains, int32_t L, double eps, int64_t iters, uint64_t seed,
                               const void* beta0, void* samples, int32_t thin, hmc_chain_stats* stats,
                               const double* temps) {
  g_last_error.clear();
  HMC_TRY(check_chains(h, chains));
  if (L < 1) return fail(HMC_EINVAL, "L must be >= 1");
  if (iters < 0) return fail(HMC_EINVAL, "iters must be >= 0");
  if (thin < 1) return fail(HMC_EINVAL, "thin must be >= 1");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(HMC_EINVAL, "eps must be finite and > 0");
  if (temps)
    for (int64_t t = 0; t < iters; ++t)
      if (!(temps[t] >= 1.0) || !std::isfinite(temps[t])) return fail(HMC_EINVAL, "every temperature must be finite and >= 1");
  const size_t sb = state_bytes(h);
  const size_t bytes = size_t(chains) * h->chain_size * sb;
  const int nprob = int(h->probs.size());

  // (Re)initialise the chain state.
  if (beta0 || h->chains_init != chains) {
    const void* b0 = nullptr;
    if (beta0) HMC_TRY(dev_in(h, 0, beta0, bytes, &b0));
    for (Problem& P : h->probs) {
      if (b0) continue;
      HMC_CUDA(cudaMemsetAsync(P.cs.beta, 0, size_t(P.state_elems) * sb, h->stream));
    }
    if (b0) HMC_TRY(pack_all(h, b0, chains, true, &StateSet::beta));
    HMC_TRY(eval_state(h, true, chains));
    for (Problem& P : h->probs) HMC_CUDA(cudaMemsetAsync(P.iter, 0, sizeof(int64_t), h->stream));
    h->chains_init = chains;
  }
  const int64_t seed_word = static_cast<int64_t>(seed);
  for (Problem& P : h->probs) {
    HMC_CUDA(cudaMemsetAsync(P.iter + 1, 0, sizeof(int64_t), h->stream));
    HMC_CUDA(cudaMemcpyAsync(P.iter + 2, &seed_word, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    HMC_CUDA(launch_init_stats(P.stats, chains, h->stream));
  }
  if (temps && iters > 0) {
    if (h->temps_cap < iters) {
      if (h->temps_d) cudaFree(h->temps_d);
      h->temps_d = nullptr;
      h->temps_cap = 0;
      HMC_CUDA(cudaMalloc(&h->temps_d, size_t(iters) * sizeof(double)));
      h->temps_cap = iters;
    }
    HMC_CUDA(cudaMemcpyAsync(h->temps_d, temps, size_t(iters) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  const int64_t nslots = samples ? iters / thin : 0;
  const size_t sample_bytes = size_t(nslots) * bytes;
  bool sh = false;
  void* sd = nullptr;
  if (samples && nslots > 0) HMC_TRY(dev_out(h, 3, samples, sample_bytes, &sd, &sh));

  if (iters > 0) {
    // One iteration as a CUDA graph, cached while its baked parameters hold.
    cudaStream_t rs_stream = h->stream ? h->stream : h->cap_stream;
    const bool use_temps = temps != nullptr;
    const bool timing = h->timing;
    if (h->gexec && !(h->g_chains == chains && h->g_L == L && h->g_eps == eps && h->g_thin == thin &&
                      h->g_samples == sd && h->g_temps == use_temps && h->g_temps_ptr == h->temps_d && h->g_timing == timing && h->g_period == h->timing_period &&
                      h->g_stream == rs_stream)) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    if (!h->gexec) {
      HMC_CUDA(cudaStreamSynchronize(h->stream));
      cudaGraph_t graph = nullptr;
      cudaStream_t cst = h->cap_stream;
      h->timer.used = 0;
      HMC_CUDA(cudaStreamBeginCapture(cst, cudaStreamCaptureModeThreadLocal));
      hmc_status cs = HMC_OK;
      std::vector<UpdateArgs> us(nprob);
      for (int b = 0; b < nprob; ++b) {
        Problem& P = h->probs[b];
        UpdateArgs u = make_update(h, P, P.cs, 0, chains, eps, b);
        u.temps = use_temps ? h->temps_d : nullptr;
        u.thin = thin;
        if (sd) {
          u.samples = static_cast<char*>(sd) + size_t(block_offset(h, b, chains)) * sb;
          u.sample_slot_stride = int64_t(chains) * h->chain_size;
        }
        us[b] = u;
        if (launch_traj_start(h->st, u, cst) != cudaSuccess) cs = fail(HMC_ECUDA, "traj_start launch failed");
      }
      for (int l = 1; l <= L && cs == HMC_OK; ++l) {
        cs = run_lpg_all(h, true, chains, cst);
        if (cs != HMC_OK) break;
        const int mode = (l < L) ? (UPD_ETA_FULL | UPD_BETA) : (UPD_ETA_HALF | UPD_SCALARS | UPD_ACCEPT);
        for (int b = 0; b < nprob && cs == HMC_OK; ++b)
          if (launch_reduce_update(h->st, us[b], mode, cst) != cudaSuccess) cs = fail(HMC_ECUDA, "reduce launch failed");
      }
      for (int b = 0; b < nprob && cs == HMC_OK; ++b)
        if (launch_select(h->st, us[b], h->probs[b].tickets + h->max_chains, cst) != cudaSuccess)
          cs = fail(HMC_ECUDA, "select launch failed");
      cudaError_t ce = cudaStreamEndCapture(cst, &graph);
      if (cs != HMC_OK) {
        if (graph) cudaGraphDestroy(graph);
        h->timer.used = 0;
        return cs;
      }
      HMC_CUDA(ce);
      ce = cudaGraphInstantiate(&h->gexec, graph, 0);
      cudaGraphDestroy(graph);
      HMC_CUDA(ce);
      h->g_chains = chains;
      h->g_L = L;
      h->g_eps = eps;
      h->g_thin = thin;
      h->g_samples = sd;
      h->g_temps = use_temps;
      h->g_temps_ptr = h->temps_d;
      h->g_timing = timing;
      h->g_period = h->timing_period;
      h->g_stream = rs_stream;
      h->g_pairs = h->timer.used;
      h->timer.used = 0;
    }
    if (rs_stream != h->stream) {
      // The private replay stream starts after the work queued on the handle's stream.
      HMC_CUDA(cudaStreamSynchronize(h->stream));
    }
    hmc_status rs = HMC_OK;
    for (int64_t t = 0; t < iters; ++t) {
      if (cudaGraphLaunch(h->gexec, rs_stream) != cudaSuccess) {
        rs = fail(HMC_ECUDA, "cudaGraphLaunch failed");
        break;
      }
      // The graph's timing events are rewritten by every replay: read them once,
      // after the last replay, so the replays run back to back (no host
      // synchronisation inside the call).
      if (timing && t == iters - 1) {
        h->timer.used = h->g_pairs;
        if ((rs = timer_harvest(h)) != HMC_OK) break;
      }
    }
    h->timer.used = 0;
    cudaStreamSynchronize(rs_stream);
    if (rs != HMC_OK) return rs;
  }
  HMC_TRY(check_device_error(h));
  if (sh) HMC_CUDA(cudaMemcpyAsync(samples, sd, sample_bytes, cudaMemcpyDeviceToHost, h->stream));
  if (stats) {
    for (int b = 0; b < nprob; ++b)
      HMC_CUDA(cudaMemcpyAsync(stats + size_t(b) * chains, h->probs[b].stats, size_t(chains) * sizeof(hmc_chain_stats),
                               cudaMemcpyDeviceToHost, h->stream));
  }
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  return HMC_OK;
}

hmc_status hmc_sample(hmc_handle h, int32_t chains, int32_t L, double eps, int64_t iters, uint64_t seed,
                      const void* beta0, void* samples, int32_t thin, hmc_chain_stats* stats) {
  return hmc_sample_tempered(h, chains, L, eps, iters, seed, beta0, samples, thin, stats, nullptr);
}

hmc_status hmc_predict(hmc_handle h, int32_t b, const void* draws, int64_t ndraws, const void* Xnew,
                       hmc_dtype x_dtype, int64_t n_new, double* prob, int32_t* cls) {
  g_last_error.clear();
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (b < 0 || b >= int(h->probs.size())) return fail(HMC_EINVAL, "problem index out of range");
  if (!draws || ndraws < 1) return fail(HMC_EINVAL, "need ndraws >= 1 coefficient draws");
  if (n_new < 0) return fail(HMC_EINVAL, "n_new must be >= 0");
  if (n_new > 0 && !Xnew) return fail(HMC_EINVAL, "Xnew is NULL");
  if (x_dtype != HMC_F64 && x_dtype != HMC_F32) return fail(HMC_EINVAL, "x_dtype must be HMC_F64 or HMC_F32");
  Problem& P = h->probs[b];
  if (P.K > predict_max_classes())
    return fail(HMC_EUNSUPPORTED, "prediction handles at most " + std::to_string(predict_max_classes()) + " classes");
  if (n_new == 0 || (!prob && !cls)) return HMC_OK;
  const size_t db = size_t(ndraws) * P.ku * P.p * state_bytes(h);
  const size_t xb = size_t(n_new) * P.p * (x_dtype == HMC_F64 ? 8 : 4);
  const void *dd = nullptr, *xd = nullptr;
  HMC_TRY(dev_in(h, 0, draws, db, &dd));
  HMC_TRY(dev_in(h, 1, Xnew, xb, &xd));
  bool ph = false, chh = false;
  void *pd = nullptr, *cd = nullptr;
  HMC_TRY(dev_out(h, 2, prob, size_t(n_new) * P.K * sizeof(double), &pd, &ph));
  HMC_TRY(dev_out(h, 3, cls, size_t(n_new) * sizeof(int32_t), &cd, &chh));
  HMC_CUDA(launch_predict(h->st, x_dtype, xd, n_new, P.p, dd, ndraws, P.ku, P.zlogit ? P.K - 1 : P.K, P.zlogit, P.K,
                          static_cast<double*>(pd), static_cast<int32_t*>(cd), h->stream));
  if (ph) HMC_CUDA(cudaMemcpyAsync(prob, pd, size_t(n_new) * P.K * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (chh) HMC_CUDA(cudaMemcpyAsync(cls, cd, size_t(n_new) * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  return HMC_OK;
}

hmc_status hmc_annealing_schedule(double t0, double r, int64_t iters, double* temps) {
  g_last_error.clear();
  if (!(t0 >= 1.0) || !std::isfinite(t0)) return fail(HMC_EINVAL, "t0 must be finite and >= 1");
  if (!(r > 0.0 && r <= 1.0)) return fail(HMC_EINVAL, "r must be in (0, 1]");
  if (iters < 0) return fail(HMC_EINVAL, "iters must be >= 0");
  if (iters > 0 && !temps) return fail(HMC_EINVAL, "temps is NULL");
  double t = t0;
  for (int64_t i = 0; i < iters; ++i) {
    t = std::max(1.0, r * t);
    temps[i] = t;
  }
  return HMC_OK;
}

hmc_status hmc_get_state(hmc_handle h, int32_t chains, void* beta, void* grad, double* logpost,
                         int64_t* next_iteration) {
  g_last_error.clear();
  HMC_TRY(check_chains(h, chains));
  const size_t bytes = size_t(chains) * h->chain_size * state_bytes(h);
  bool bh = false, gh = false, lh = false;
  void *bd = nullptr, *gd = nullptr, *ld = nullptr;
  HMC_TRY(dev_out(h, 0, beta, bytes, &bd, &bh));
  HMC_TRY(dev_out(h, 1, grad, bytes, &gd, &gh));
  HMC_TRY(dev_out(h, 2, logpost, h->probs.size() * chains * sizeof(double), &ld, &lh));
  if (bd) HMC_TRY(unpack_all(h, bd, chains, true, &StateSet::beta));
  if (gd) HMC_TRY(unpack_all(h, gd, chains, true, &StateSet::grad));
  if (ld) HMC_TRY(copy_logk(h, static_cast<double*>(ld), chains, 0));
  if (bh) HMC_CUDA(cudaMemcpyAsync(beta, bd, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (gh) HMC_CUDA(cudaMemcpyAsync(grad, gd, bytes, cudaMemcpyDeviceToHost, h->stream));
  if (lh)
    HMC_CUDA(cudaMemcpyAsync(logpost, ld, h->probs.size() * chains * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (next_iteration)
    HMC_CUDA(cudaMemcpyAsync(next_iteration, h->probs[0].iter, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  return HMC_OK;
}

// ------------------------------------------------------------- checkpoints
// File layout (host byte order): the 8 bytes "HMCCKPT2"; int32 state type,
// number of problems, chains, X storage type, prior kind, coefficient layout;
// double prior scale; per problem int64 n, int32 p, int32 K, int64 next global
// iteration; then beta and grad of every chain in the beta layout of
// hmc_logpost_grad (state type), and log K as double[nprob * chains].
namespace {
constexpr char kCkptMagic[8] = {'H', 'M', 'C', 'C', 'K', 'P', 'T', '2'};
struct FileCloser {
  FILE* f = nullptr;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};

// Largest |a - b| / max(1, |b|) over n doubles, and the relative 2-norm error
// ||a - b|| / ||b|| over n values of the state type (bytes per value sb).
double logk_mismatch(const double* a, const double* b, size_t n) {
  double m = 0.0;
  for (size_t i = 0; i < n; ++i) {
    const double d = std::fabs(a[i] - b[i]) / std::max(1.0, std::fabs(b[i]));
    m = std::max(m, std::isfinite(d) ? d : 1e300);
  }
  return m;
}
double grad_mismatch(const char* a, const char* b, size_t n, size_t sb) {
  double num = 0.0, den = 0.0;
  for (size_t i = 0; i < n; ++i) {
    double x, y;
    if (sb == 8) {
      std::memcpy(&x, a + i * 8, 8);
      std::memcpy(&y, b + i * 8, 8);
    } else {
      float xf, yf;
      std::memcpy(&xf, a + i * 4, 4);
      std::memcpy(&yf, b + i * 4, 4);
      x = xf;
      y = yf;
    }
    num += (x - y) * (x - y);
    den += y * y;
  }
  const double r = std::sqrt(num) / std::max(std::sqrt(den), 1e-300);
  return std::isfinite(r) ? r : 1e300;
}
}  // namespace

hmc_status hmc_state_save(hmc_handle h, const char* path) {
  g_last_error.clear();
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (!path) return fail(HMC_EINVAL, "path is NULL");
  const int chains = h->chains_init;
  if (chains < 1) return fail(HMC_EINVAL, "no chain state to save: run hmc_sample first");
  const int nprob = int(h->probs.size());
  const size_t bytes = size_t(chains) * h->chain_size * state_bytes(h);
  std::vector<char> hb(bytes), hg(bytes);
  std::vector<double> hl(size_t(nprob) * chains);
  std::vector<int64_t> it(nprob);
  void* d = nullptr;
  HMC_TRY(grow_staging(h, 0, bytes, &d));
  HMC_TRY(unpack_all(h, d, chains, true, &StateSet::beta));
  HMC_CUDA(cudaMemcpyAsync(hb.data(), d, bytes, cudaMemcpyDeviceToHost, h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));   // the staging buffer takes grad next
  HMC_TRY(unpack_all(h, d, chains, true, &StateSet::grad));
  HMC_CUDA(cudaMemcpyAsync(hg.data(), d, bytes, cudaMemcpyDeviceToHost, h->stream));
  for (int b = 0; b < nprob; ++b) {
    HMC_CUDA(cudaMemcpyAsync(hl.data() + size_t(b) * chains, h->probs[b].logk, size_t(chains) * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
    HMC_CUDA(cudaMemcpyAsync(&it[b], h->probs[b].iter, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  }
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  FileCloser fc;
  fc.f = std::fopen(path, "wb");
  if (!fc.f) return fail(HMC_EINVAL, std::string("cannot open ") + path + " for writing");
  const int32_t hdr[6] = {int32_t(h->st), int32_t(nprob), int32_t(chains), int32_t(h->xt), int32_t(h->prior_kind),
                          int32_t(h->layout)};
  bool ok = std::fwrite(kCkptMagic, 1, 8, fc.f) == 8 && std::fwrite(hdr, sizeof(int32_t), 6, fc.f) == 6 &&
            std::fwrite(&h->prior_scale, sizeof(double), 1, fc.f) == 1;
  for (int b = 0; b < nprob && ok; ++b) {
    const Problem& P = h->probs[b];
    const int64_t n = P.n;
    const int32_t pk[2] = {P.p, P.K};
    ok = std::fwrite(&n, sizeof(int64_t), 1, fc.f) == 1 && std::fwrite(pk, sizeof(int32_t), 2, fc.f) == 2 &&
         std::fwrite(&it[b], sizeof(int64_t), 1, fc.f) == 1;
  }
  ok = ok && std::fwrite(hb.data(), 1, bytes, fc.f) == bytes && std::fwrite(hg.data(), 1, bytes, fc.f) == bytes &&
       std::fwrite(hl.data(), sizeof(double), hl.size(), fc.f) == hl.size();
  const int closed = std::fclose(fc.f);
  fc.f = nullptr;
  if (!ok || closed != 0) return fail(HMC_EINVAL, std::string("writing ") + path + " failed");
  return HMC_OK;
}

hmc_status hmc_state_load(hmc_handle h, const char* path) {
  g_last_error.clear();
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (!path) return fail(HMC_EINVAL, "path is NULL");
  FileCloser fc;
  fc.f = std::fopen(path, "rb");
  if (!fc.f) return fail(HMC_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[6];
  double pscale = 0.0;
  if (std::fread(magic, 1, 8, fc.f) != 8 || std::memcmp(magic, kCkptMagic, 8) != 0 ||
      std::fread(hdr, sizeof(int32_t), 6, fc.f) != 6 || std::fread(&pscale, sizeof(double), 1, fc.f) != 1)
    return fail(HMC_EINVAL, std::string(path) + " is not a chain-state checkpoint");
  const int nprob = int(h->probs.size());
  if (hdr[0] != h->st) return fail(HMC_EINVAL, "the checkpoint's state type differs from the handle's");
  if (hdr[1] != nprob) return fail(HMC_EINVAL, "the checkpoint holds a different number of problems");
  if (hdr[3] != h->xt) return fail(HMC_EINVAL, "the checkpoint was taken with another storage type of X");
  if (hdr[4] != h->prior_kind || pscale != h->prior_scale)
    return fail(HMC_EINVAL, "the checkpoint was taken under another prior (kind or scale)");
  if (hdr[5] != h->layout) return fail(HMC_EINVAL, "the checkpoint uses another coefficient layout");
  const int chains = hdr[2];
  if (chains < 1 || chains > h->max_chains)
    return fail(HMC_EINVAL, "the checkpoint's chain count is outside [1, max_chains]");
  std::vector<int64_t> it(nprob);
  for (int b = 0; b < nprob; ++b) {
    int64_t n = 0;
    int32_t pk[2] = {0, 0};
    if (std::fread(&n, sizeof(int64_t), 1, fc.f) != 1 || std::fread(pk, sizeof(int32_t), 2, fc.f) != 2 ||
        std::fread(&it[b], sizeof(int64_t), 1, fc.f) != 1)
      return fail(HMC_EINVAL, std::string(path) + " is truncated");
    const Problem& P = h->probs[b];
    if (n != P.n || pk[0] != P.p || pk[1] != P.K)
      return fail(HMC_EINVAL, "problem " + std::to_string(b) + " of the checkpoint has another shape (n, p, K)");
    if (it[b] < 0) return fail(HMC_EINVAL, "negative iteration index in the checkpoint");
  }
  const size_t sb = state_bytes(h);
  const size_t bytes = size_t(chains) * h->chain_size * sb;
  std::vector<char> hb(bytes), hg(bytes), rg(bytes);
  std::vector<double> hl(size_t(nprob) * chains), rl(hl.size());
  if (std::fread(hb.data(), 1, bytes, fc.f) != bytes || std::fread(hg.data(), 1, bytes, fc.f) != bytes ||
      std::fread(hl.data(), sizeof(double), hl.size(), fc.f) != hl.size())
    return fail(HMC_EINVAL, std::string(path) + " is truncated");
  // The saved gradient and log K are reused as the state of the next
  // trajectory's first half step and accept test, so they must belong to this
  // handle's posterior: evaluate both at the saved coefficients (user scratch
  // state, the chain state is untouched) and compare.  The same X, labels and
  // prior agree to rounding order; another posterior does not.
  void* d = nullptr;
  HMC_TRY(grow_staging(h, 0, bytes, &d));
  HMC_CUDA(cudaMemcpyAsync(d, hb.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  HMC_TRY(pack_all(h, d, chains, false, &StateSet::beta));
  HMC_TRY(eval_state(h, false, chains));
  HMC_TRY(unpack_all(h, d, chains, false, &StateSet::grad));
  HMC_CUDA(cudaMemcpyAsync(rg.data(), d, bytes, cudaMemcpyDeviceToHost, h->stream));
  for (int b = 0; b < nprob; ++b)
    HMC_CUDA(cudaMemcpyAsync(rl.data() + size_t(b) * chains, h->probs[b].logk + h->max_chains,
                             size_t(chains) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HMC_TRY(check_device_error(h));
  const double el = logk_mismatch(hl.data(), rl.data(), hl.size());
  const double eg = grad_mismatch(hg.data(), rg.data(), bytes / sb, sb);
  const double tol = h->xt == HMC_F64 ? 1e-9 : 1e-4;
  if (el > tol || eg > tol) {
    char buf[200];
    std::snprintf(buf, sizeof(buf),
                  "the checkpoint does not belong to this handle's posterior (log K mismatch %.3g, gradient "
                  "mismatch %.3g at the saved coefficients; tolerance %.0e)", el, eg, tol);
    return fail(HMC_EINVAL, buf);
  }
  HMC_CUDA(cudaMemcpyAsync(d, hb.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  HMC_TRY(pack_all(h, d, chains, true, &StateSet::beta));
  HMC_CUDA(cudaMemcpyAsync(d, hg.data(), bytes, cudaMemcpyHostToDevice, h->stream));   // after the pack, in stream order
  HMC_TRY(pack_all(h, d, chains, true, &StateSet::grad));
  for (int b = 0; b < nprob; ++b) {
    HMC_CUDA(cudaMemcpyAsync(h->probs[b].logk, hl.data() + size_t(b) * chains, size_t(chains) * sizeof(double),
                             cudaMemcpyHostToDevice, h->stream));
    HMC_CUDA(cudaMemcpyAsync(h->probs[b].iter, &it[b], sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  }
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  h->chains_init = chains;
  return HMC_OK;
}

hmc_status hmc_get_x(hmc_handle h, int32_t b, void* dst, float* scales) {
  g_last_error.clear();
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (b < 0 || b >= int(h->probs.size())) return fail(HMC_EINVAL, "problem index out of range");
  if (!dst) return fail(HMC_EINVAL, "dst is NULL");
  Problem& P = h->probs[b];
  const size_t xb = dtype_bytes(h->xt);
  if (P.n > 0 && (P.engine == 2 || P.engine == 3)) {
    void* tmp = nullptr;
    HMC_CUDA(cudaMalloc(&tmp, size_t(P.n) * P.p * xb));
    cudaError_t e = tc_tiles_to_rows(P.X, tmp, P.n, P.p, P.p_pad, h->xt == HMC_FP8E4M3, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, size_t(P.n) * P.p * xb, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    HMC_CUDA(e);
  } else if (P.n > 0) {
    HMC_CUDA(cudaMemcpy2DAsync(dst, size_t(P.p) * xb, P.X, size_t(P.p_pad) * xb, size_t(P.p) * xb, size_t(P.n),
                               cudaMemcpyDefault, h->stream));
  }
  if (scales && P.xscale)
    HMC_CUDA(cudaMemcpyAsync(scales, P.xscale, size_t(P.p) * sizeof(float), cudaMemcpyDefault, h->stream));
  HMC_CUDA(cudaStreamSynchronize(h->stream));
  return HMC_OK;
}

const char* hmc_describe(hmc_handle h) { return h ? h->desc.c_str() : "{}"; }

hmc_status hmc_set_timing(hmc_handle h, int32_t enable) {
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  h->timing = enable != 0;
  h->timing_period = enable > 1 ? enable : 1;
  h->timing_seq = 0;
  h->timing_ms = 0.0;
  h->timing_first_ms = 0.0;
  h->timing_launches = 0;
  h->timer.used = 0;
  return HMC_OK;
}

hmc_status hmc_fused_kernel_time(hmc_handle h, double* total_ms, int64_t* launches) {
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (total_ms) *total_ms = h->timing_ms;
  if (launches) *launches = h->timing_launches;
  return HMC_OK;
}

hmc_status hmc_first_pass_time(hmc_handle h, double* first_ms) {
  if (!h) return fail(HMC_EINVAL, "NULL handle");
  if (first_ms) *first_ms = h->timing_first_ms;
  return HMC_OK;
}

}  // extern "C"
