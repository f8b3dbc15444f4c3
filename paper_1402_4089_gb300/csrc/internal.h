// Host-side declarations shared by the translation units of libhmc.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/hmc.h"

namespace hmc {

// One launch of a fused log-posterior/gradient pass (Eqs. logkernel and
// gradient): every cluster of S CTAs walks row tiles of BM rows; CTA `rank`
// of a cluster owns the column slice [rank*PC, (rank+1)*PC) of X and of the
// coefficients.  Outputs are per-cluster partial sums reduced later in a
// fixed order (no floating-point atomics).
struct LpgArgs {
  const void* X;            // [n][p_pad] storage type, zero-padded columns
  const int32_t* y;         // [n]
  const float* xscale;      // [p_pad] FP8 column scales, or nullptr
  const void* beta;         // [C][p_pad] state type (first column of this launch)
  void* gpart;              // partial gradient, state type; cluster b at gpart + b*gpart_cstride
  int64_t gpart_cstride;    // elements between consecutive clusters' partials
  double* lpart;            // partial log-likelihood per chain; cluster b at lpart + b*lpart_cstride
  int32_t lpart_cstride;
  int* err;                 // device error word (bits of hmc::ERR_*)
  int64_t n;                // rows
  int32_t p_pad;            // padded columns (= S * PC)
  int32_t PC;               // columns per CTA
  int32_t C;                // coefficient columns of this launch (chains * Km1)
  int32_t Km1;              // free coefficient rows per chain (K - 1, or K when unconstrained)
  int32_t zlogit;           // 1: class K is the implied zero logit (valid labels 0..Km1); 0: none (0..Km1-1)
  int32_t chains;           // chains of this launch
  int32_t BM;               // rows per super-tile (8 on the CUDA-core engine)
  int32_t CR;               // unused by the CUDA-core engine (kept equal to BM)
  int32_t S;                // cluster size
  int32_t NT;               // threads per CTA (consumer warps + 1 producer warp)
  int32_t NSTAGE;           // ring slots (super-tiles) in shared memory
  int32_t nclusters;        // clusters in the grid
  int64_t ntiles;           // ceil(n / BM)
  long long spin_limit;     // probes per bounded wait
  int32_t inject_timeout;   // 1: wait on a barrier nothing arrives at (host-side fault injection)
  int32_t NWL;              // CUDA-core engine: logit warps (the rest but one are gradient warps)
};

// CUDA-core fused kernel (any X storage type, small C).
constexpr int kSimtMaxThreads = 512;   // up to 10 gradient + 5 logit + 1 producer warps
constexpr int kSimtRows = 16;          // rows per super-tile of the CUDA-core kernel (host and device)
int simt_max_ct(int xt);                                     // largest C one launch handles
// Shared memory of one CTA: PC columns, cluster size S, NWL logit warps, NSTAGE ring slots.
size_t simt_smem_bytes(int xt, int st, int C, int PC, int S, int NWL, int NSTAGE);
cudaError_t simt_prepare(int xt, int st, int C, size_t smem, int S);   // func attributes
// Tile of the CUDA-core pass: cluster size S (CTA column slice PC, a multiple
// of 16), NWC gradient warps (one per 32 column quads), NWL logit warps,
// NSTAGE ring slots; NT = 32 * (NWC + NWL + 1) threads.
struct SimtTile {
  int S, PC, NWC, NWL, NT, NSTAGE;
  size_t smem;
  int maxclu;   // clusters resident at once
};
// Picks the tile keeping the most SMs streaming X (S = 0 in *out: none fits).
// force_S / force_NS: 0 = free.  exact_ld > 0: S * PC must equal it.
cudaError_t simt_choose(int xt, int C, int64_t p, int64_t ntiles, int force_S, int force_NS, int64_t exact_ld,
                        SimtTile* out);
cudaError_t simt_max_active_clusters(int xt, int st, int C, size_t smem, int S, int NT, int* out);
// C_kernel: the column bound the handle was prepared for (a smaller last chain group
// still runs that instantiation).
cudaError_t simt_launch(int xt, int st, const LpgArgs& a, size_t smem, cudaStream_t stream, int C_kernel);
int simt_ct_of(int xt, int C);                               // class bound of the kernel serving C columns
int simt_max_grad_warps(int xt, int C);                      // gradient warps the kernel allows
int simt_logit_warps(int nwc);                               // logit warps paired with nwc gradient warps
// One launch for several problems (table and first on the device; first has nprob + 1 entries).
cudaError_t simt_prepare_batched(int xt, int C, int S);
cudaError_t simt_max_active_clusters_batched(int xt, int C, size_t smem, int S, int NT, int* out);
cudaError_t simt_launch_batched(int xt, int C, const LpgArgs* table, const int* first, int nprob, int chains,
                                int total_clusters, int S, int NT, size_t smem, cudaStream_t stream);

// Tensor-core fused kernel (BF16 or FP8 X, tcgen05 + TMEM + bulk copies), lpg_tc.cu.
struct TcPlan {
  int N, NP, PC, MB, S;
  uint32_t tmem_cols, stage_bytes;
  int nz = 1;      // logit accumulators in TMEM
  int slots = 1;   // partial-logit receive slots
  int rbufs = 1;   // R operand buffers
  int la = 1;      // lookahead (tiles) between the two sweeps
};
constexpr int kTcMaxDepth = 4;
struct TcLaunch {
  const void* xs;           // X boxes (tc_x_to_tiles / tc_x_to_tiles_fp8 layout)
  const float* xscale;      // FP8 column scales (nullptr for BF16)
  int32_t fp8;
  const void* bs;           // coefficient operand boxes (tc_beta_to_tiles layout)
  int64_t n;
  int32_t p_pad, C, Km1, chains, NST, nclusters;
  void* gpart;
  int64_t gpart_cstride;
  double* lpart;
  int32_t lpart_cstride;
  const int32_t* y;
  int* err;
  long long spin_limit;
  int32_t inject_timeout;
  int32_t zlogit;           // 1: class K is the implied zero logit; 0: all Km1 classes free
};
bool tc_plan(int64_t p, int C, int S, TcPlan* out);
size_t tc_smem_bytes(const TcPlan& pl, int NST, int chains, bool fp8);
int tc_threads(bool fp8);                   // threads of one CTA (FP8 adds converter warps)
cudaError_t tc_prepare(size_t smem, int S, bool fp8);
cudaError_t tc_max_active_clusters(size_t smem, int S, bool fp8, int* out);
cudaError_t tc_x_to_tiles(int in_dtype, const void* X, void* out, int64_t n, int32_t p, int32_t p_pad, int* err,
                          cudaStream_t s);
cudaError_t tc_x_to_tiles_fp8(int in_dtype, const void* X, const float* scales, void* out, int64_t n, int32_t p,
                              int32_t p_pad, int* err, cudaStream_t s);
cudaError_t tc_tiles_to_rows(const void* tiles, void* out_bits, int64_t n, int32_t p, int32_t p_pad, bool fp8,
                             cudaStream_t s);
cudaError_t tc_beta_to_tiles(const float* beta, const float* scales, void* out, int C, int N, int p_pad,
                             cudaStream_t s);
cudaError_t tc_launch(const TcPlan& pl, const TcLaunch& L, size_t smem, cudaStream_t stream);
// One launch for several problems (shared cluster size and storage type).
struct TcBetaBox {
  const float* beta;        // [chains][Km1][p_pad] state
  const float* scales;      // FP8 column scales or nullptr
  void* out;                // operand boxes of the problem
  int32_t Km1, N, p_pad;
};
cudaError_t tc_prepare_batched(size_t smem, int S, bool fp8);
cudaError_t tc_max_active_clusters_batched(size_t smem, int S, bool fp8, int* out);
cudaError_t tc_upload_batch(const TcPlan* plans, const TcLaunch* launches, int m, void** d_table);
cudaError_t tc_upload_beta_table(const TcBetaBox* boxes, int m, void** d_table);
int tc_beta_job_bytes();                    // bytes of one coefficient-box job in the device table
cudaError_t tc_beta_to_tiles_batched(const void* d_table, int m, int chains, int64_t max_elems, cudaStream_t s);
cudaError_t tc_launch_batched(const void* d_table, const int* d_first, int m, int chains, int total_clusters, int S,
                              bool fp8, size_t smem, cudaStream_t stream);

// Two-pass tensor-core engine (BF16 X), lpg_tc2.cu: pass A forms the logits,
// softmax and residual R of every (row tile, chain group) unit, pass B the
// partial gradients X^T R of every (feature group, chain group, row range) unit.
struct Tc2Plan {
  int p_pad = 0;            // p rounded to 128
  int gc = 0, N = 0, NB = 0;  // chains per group, MMA N (>= gc (K-1), multiple of 16), R boxes (64 columns)
  int gridA = 0, nstA = 0;  // pass A CTAs and ring slots
  int U = 1;                // pass A row tiles per unit (sharing each coefficient box)
  size_t smemA = 0;
  int MB = 0, nfg = 0, Q = 0;   // pass B: 128-feature blocks per CTA, feature groups, row ranges
  int nstB = 0, nrsB = 0;   // pass B X ring slots and R slots
  size_t smemB = 0;
};
struct Tc2Launch {
  const void* xs;           // X boxes (tc_x_to_tiles layout with p_pad columns; FP8: tc_x_to_tiles_fp8)
  const float* xscale;      // FP8: per-column scales (folded into the gradient); else unused
  int32_t fp8;              // X boxes hold FP8 E4M3 codes
  const void* bs;           // coefficient operand of every group (tc2_beta_boxes)
  const int32_t* y;
  void* rbuf;               // R boxes [ntiles][groups][NB][16 KB]
  void* spart;              // [gridA][U][N][128] FP32 partial logits of units split over two CTAs
  int* sflag;               // [gridA] partial-ready flags (zero between launches)
  double* lpart;            // [gridA][lpart_cstride]
  int32_t lpart_cstride;
  void* gpart;              // [Q][chains Km1][p_pad] FP32
  int64_t gpart_cstride;
  int* err;
  int64_t n;
  int32_t Km1, zlogit, chains;
  long long spin_limit;
};
// force_U: 0, or the row tiles per pass-A unit to use (false if they do not fit).
bool tc2_plan(int64_t n, int64_t p, int Km1, int chains, int nsm, int smem_max, int force_U, Tc2Plan* out);
int tc2_threads(bool fp8);
cudaError_t tc2_prepare();
// scales: FP8 column scales folded into the coefficients, or nullptr.
cudaError_t tc2_beta_boxes(const float* beta, const float* scales, void* out, int Km1, int gc, int chains, int N,
                           int p_pad, int ngroups, cudaStream_t s);
// `between` (or nullptr): an event recorded between the two passes (a graph node when capturing).
cudaError_t tc2_launch(const Tc2Plan& P, const Tc2Launch& L, cudaStream_t stream, cudaEvent_t between, bool capturing);

// Two-pass CUDA-core engine (FP64 / FP32 X), lpg_simt2.cu: for shapes the fused
// CUDA-core pass cannot tile.  X row-major [n][p_pad] (p_pad a multiple of 4).
struct Simt2Launch {
  const void* X;
  const int32_t* y;
  const float* xscale;      // nullptr (scales are folded into X for these storage types)
  const void* beta;         // [C][p_pad] state type
  void* rbuf;               // [n][C] residuals (state type)
  void* zpart;              // [FS][n][C] partial logits of the feature splits (state type)
  double* lrow;             // [ceil(n / 8)][lrow_stride] log-likelihoods of 8-row blocks, chains of this launch first
  int32_t lrow_stride;
  void* gpart;              // [Q][C][p_pad] state type
  int64_t gpart_cstride;
  int* err;
  int64_t n;
  int32_t p_pad, C, Km1, chains, zlogit, Q, FS;
};
int simt2_max_c();
int64_t simt2_ll_blocks(int64_t n);   // log-likelihood partials per chain
int simt2_row_ranges(int64_t n, int32_t p_pad, int32_t C, int nsm);
int simt2_feature_splits(int64_t n, int32_t p_pad, int nsm);
cudaError_t simt2_prepare(int xt);
// `between` (optional) is recorded after the first pass (as an external node
// when the stream is capturing).
cudaError_t simt2_launch(int xt, const Simt2Launch& L, cudaStream_t s, cudaEvent_t between, bool capturing);

// Element-wise / reduction kernels (update.cu).
struct UpdateArgs {
  void* beta;  void* eta;  void* grad;          // [chains][Km1][p_pad] state type
  void* beta0; void* grad0;                     // saved trajectory start
  const void* gpart; int64_t gpart_cstride; int32_t nparts;   // partial gradients
  int32_t glanes;   // lanes sharing one coefficient's partial sum (power of two <= 32; 0 or 1: one)
  const double* lpart; int32_t lpart_cstride; int32_t nlparts; // partial log-likelihoods
  double* logk;     // [chains] current log K
  void* ugrad;      // optional: the gradient also written in the user layout [chains][ku][p] (masked row zero)
  double* ulogk;    // optional: log K also written here [chains]
  double* logk0;    // [chains] at trajectory start
  double* h0;       // [chains] H at trajectory start
  double* scal;     // scratch [chains][nblk][2] block partials
  unsigned int* tickets;  // [chains] last-block counters (self-resetting)
  int* accept;      // [chains]
  void* stats;      // [chains] hmc_chain_stats (device)
  const double* temps;  // [iters] or nullptr
  int64_t* iter;    // device iteration counter (global, for the RNG)
  int64_t* local_iter; // iteration within the current hmc_sample call
  void* samples; int32_t thin; int64_t sample_slot_stride;  // user layout: [slot][...][chains][Km1][p]
  int32_t chains_word_hi;  // problem index (high half of the RNG chain word)
  int* err;
  int32_t p, p_pad, Km1, chains, nblk;
  int32_t ku;       // rows per chain of the user layout (samples): Km1, or Km1 + 1 with a zero masked row
  int32_t prior_kind; double prior_scale;
  double eps;
  const uint64_t* seed;  // device: generator key of the current hmc_sample call
};

enum : int {
  UPD_ETA_HALF = 1,     // eta += eps/2 * g
  UPD_ETA_FULL = 2,     // eta += eps * g
  UPD_BETA = 4,         // beta += eps * eta (after the eta update)
  UPD_SCALARS = 8,      // log K (and kinetic energy) per chain
  UPD_ACCEPT = 16,      // end of trajectory: Metropolis test
};

cudaError_t launch_reduce_update(int st, const UpdateArgs& a, int mode, cudaStream_t s);
cudaError_t launch_traj_start(int st, const UpdateArgs& a, cudaStream_t s);
cudaError_t launch_select(int st, const UpdateArgs& a, unsigned int* ticket_all, cudaStream_t s);
int update_blocks_per_chain(int64_t per_chain);   // per_chain: coefficients x group lanes
int update_group_lanes(int64_t per_chain, int chains, int nparts, int nsm);
cudaError_t launch_leap_start(int st, const UpdateArgs& a, cudaStream_t s);

// Layout conversion between the user layout [chains][ku][p] (state type)
// and the padded device layout [chains][km1][p_pad] (ku >= km1): pack drops
// rows km1..ku-1 of each chain (a masked row), unpack writes them as zero.
cudaError_t launch_pack(int st, const void* src, void* dst, int64_t chains, int32_t ku, int32_t km1, int32_t p,
                        int32_t p_pad, cudaStream_t s);
cudaError_t launch_unpack(int st, const void* src, void* dst, int64_t chains, int32_t ku, int32_t km1, int32_t p,
                          int32_t p_pad, cudaStream_t s);

// X upload: convert float/double rows into the storage type with padding.
cudaError_t launch_convert_x(int in_dtype, const void* src, int xt, void* dst, const float* scales, int64_t n, int32_t p,
                             int32_t p_pad, int* err, cudaStream_t s);
cudaError_t launch_fp8_scales(int in_dtype, const void* src, float* scales, int64_t n, int32_t p, int32_t p_pad,
                              cudaStream_t s);
cudaError_t launch_check_labels(const int32_t* y, int64_t n, int32_t K, int* err, cudaStream_t s);
cudaError_t launch_init_stats(void* stats, int chains, cudaStream_t s);

// Posterior predictive (predict.cu): mean softmax over `ndraws` coefficient
// draws [ndraws][ku][p] (state type) for the rows of X (n x p, in_dtype), and
// its argmax.  K <= predict_max_classes().
int predict_max_classes();
cudaError_t launch_predict(int st, int in_dtype, const void* X, int64_t n, int32_t p, const void* draws, int64_t ndraws,
                           int32_t ku, int32_t km1, int32_t zlogit, int32_t K, double* prob, int32_t* cls,
                           cudaStream_t s);

// Message returned by hmc_last_error() for the calling thread.
void set_last_error(const std::string& msg);

}  // namespace hmc
