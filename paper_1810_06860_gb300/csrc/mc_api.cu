// Host orchestration and C ABI of the GB300 fast-SVT library.
//
//   rSVD-BKI (Alg. 5) and rSVD-PI (Alg. 4) on the device-resident sparse
//   iterate; the SVT iteration of Alg. 6 with subspace recycling (Sec. IV.B)
//   and the adaptive power parameter.  Control decisions (the repeat test, the
//   rank r, p adaptation, the stopping test) are taken on the host in float64
//   from a few scalars copied back per SVD call; everything else runs in the
//   kernels of k_rng.cu, k_sparse.cu and k_dense.cu.
//
// The block-Krylov basis is built block by block: every new block
// A (A^T Q_{i-1}) is projected against the previous blocks twice and then
// normalised by CholeskyQR (shifted first pass, then two plain passes).  The
// union of the blocks spans the same space as [H_0 ... H_p] of Alg. 5, so by
// Lemma 2 (any orthonormal basis of the range) and Lemma 3 (lu() only
// rescales within that range) the result is the paper's, computed with a
// better-conditioned basis in float32.
#include "mc_common.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

namespace mc {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_error(const std::string &msg) { g_last_error = msg; }
[[noreturn]] void fail(mc_status st, const std::string &msg) { throw Err{st, msg}; }

void *Alloc::get(size_t bytes) {
  if (bytes == 0) bytes = 256;
  void *p = nullptr;
  if (has_hook) {
    p = hook.alloc(hook.ctx, bytes, stream);
    if (!p) fail(MC_ENOMEM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    const cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(MC_ENOMEM, "cudaMallocAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  return p;
}

void Alloc::put(void *p, size_t bytes) {
  if (!p) return;
  if (has_hook) hook.free(hook.ctx, p, bytes, stream);
  else cudaFreeAsync(p, stream);
}

void DBuf::reserve(Alloc &a, size_t bytes) {
  if (bytes <= cap && p) return;
  release(a);
  p = a.get(bytes);
  cap = bytes;
}

void DBuf::release(Alloc &a) {
  if (p) a.put(p, cap);
  p = nullptr;
  cap = 0;
}

}  // namespace mc

using namespace mc;

namespace {

constexpr int kMaxKt = 1024;  // widest Krylov basis the small eigensolver takes

// CUDA-event timing of kernel classes on the handle's stream (off by default).
struct Prof {
  bool on = false;
  unsigned mask = ~0u;  // kernel classes recorded while on
  struct Rec {
    int cat;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  mc_timing acc[MC_T_COUNT] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    MC_CUDA(cudaEventCreate(&e));
    return e;
  }
  void resolve() {
    for (auto &r : pending) {
      float ms = 0.f;
      MC_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      acc[r.cat].ms += ms;
      acc[r.cat].bytes += r.bytes;
      acc[r.cat].flops += r.flops;
      acc[r.cat].launches += 1;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  void reset() {
    for (auto &r : pending) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
    for (auto &a : acc) a = mc_timing{};
  }
  ~Prof() {
    for (auto &r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct mc_handle_s {
  int64_t m = 0, n = 0, nnz = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // side stream for the copy of Y into CSC order after an update: it
  // overlaps the residual read-back, the host decisions and the start of the
  // next step; readers of the CSC copy wait for ev_yc first
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_yc = nullptr;
  bool yc_pending = false;
  bool single_stream = false;  // the copy stays on the main stream
  Alloc alloc;
  // CSR (rix: row of every entry)
  DBuf rp, ci, mval, y, rix;
  // CSC
  DBuf cp, ri, perm, yc;
  SegPlan plan_r, plan_c;
  // panels
  DBuf Om, Q, H, Tmp, T, Bt, G, C, Rinv, lam, W, Wsel, scale, U, V, Ub, Vb, seg_sq, dsum, tn_part, sp_part, eig_work;
  DBuf Om_bf, Q_bf, T_bf;  // bf16 panels of the mixed-precision form
  int precision = 0;       // 0 plain float32, 1 bf16 panels in the Krylov products
  DBuf flags;
  // rSVD result bookkeeping
  int Kq = 0;          // columns of the basis whose Ritz pairs are in W (incl. zero padding)
  int bt_ready = 0;    // leading columns of Bt = Y^T Q already formed by the Krylov loop
  int q_real = 0;      // real (non-padding) columns of the stored Krylov basis
  int kw = 0;          // eigenpairs in lam/W
  std::vector<float> h_lam;
  // pinned staging of small host-to-device parameter copies: two slots used
  // in turn, each with an event marking when its last copy has run
  float *h_stage[2] = {nullptr, nullptr};
  size_t h_stage_cap[2] = {0, 0};
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  int stage_next = 0;
  // SVT state
  bool svt_init = false;
  mc_params prm{};
  double tau = 0, normF = 0, norm2 = 0, c = 0;
  int it = 0, r = 0, q = 0, p = 3, streak = 0;
  double prev_err = std::numeric_limits<double>::infinity();
  uint64_t call_id = 1;
  int basis = 0;       // 0 none, 1 Q in this->Q (q_real columns), 2 U in this->Ub (ub_k columns)
  int ub_k = 0, ub_ld = 0;
  int vb_k = 0, vb_ld = 0;  // previous right singular vectors (warm start)
  std::vector<double> sig;  // singular values of the last SVD (descending)
  int us_ld = 4;       // leading dim of U / V (shrunk factors) of the estimate
  int r_cur = 0;       // columns of the current estimate
  std::vector<float> h_sig_r;
  double last_err = 0;
  Prof prof;
};


namespace mc {
void handle_single_stream(mc_handle h) {
  if (h) h->single_stream = true;
}
}  // namespace mc

namespace {

// ------------------------------------------------------------------ helpers --
void copy_in(cudaStream_t st, void *dst, const void *src, size_t bytes) {
  if (bytes == 0) return;
  MC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}

void copy_out_2d(cudaStream_t st, float *dst, int dst_cols, const float *src, int src_ld, int64_t rows) {
  if (!dst || rows <= 0 || dst_cols <= 0) return;
  MC_CUDA(cudaMemcpy2DAsync(dst, sizeof(float) * dst_cols, src, sizeof(float) * src_ld, sizeof(float) * dst_cols, rows,
                            cudaMemcpyDefault, st));
}

void sync(mc_handle h) { MC_CUDA(cudaStreamSynchronize(h->stream)); }

}  // namespace

bool mc::use_pdl() {
  static const bool on = [] {
    const char *v = std::getenv("MC_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

void mc::smem_attr(const void *fn, int bytes) {
  static std::mutex mu;
  static std::vector<std::tuple<const void *, int, int>> done;  // (kernel, device, bytes)
  int dev = 0;
  MC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  for (const auto &d : done)
    if (std::get<0>(d) == fn && std::get<1>(d) == dev && std::get<2>(d) >= bytes) return;
  MC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.emplace_back(fn, dev, bytes);
}

namespace {

// count floats from host memory to dst (device) on the handle's stream,
// through a pinned slot: returns without waiting for the copy; a slot is
// rewritten only after its previous copy has run
void stage_copy(mc_handle h, float *dst, const float *src, size_t count) {
  if (count == 0) return;
  const int s = h->stage_next;
  h->stage_next ^= 1;
  if (h->stage_ev[s]) MC_CUDA(cudaEventSynchronize(h->stage_ev[s]));
  else MC_CUDA(cudaEventCreateWithFlags(&h->stage_ev[s], cudaEventDisableTiming));
  if (h->h_stage_cap[s] < count) {
    if (h->h_stage[s]) MC_CUDA(cudaFreeHost(h->h_stage[s]));
    h->h_stage[s] = nullptr;
    h->h_stage_cap[s] = 0;
    const size_t cap = std::max<size_t>(count, 256);
    MC_CUDA(cudaMallocHost(reinterpret_cast<void **>(&h->h_stage[s]), sizeof(float) * cap));
    h->h_stage_cap[s] = cap;
  }
  std::memcpy(h->h_stage[s], src, sizeof(float) * count);
  MC_CUDA(cudaMemcpyAsync(dst, h->h_stage[s], sizeof(float) * count, cudaMemcpyHostToDevice, h->stream));
  MC_CUDA(cudaEventRecord(h->stage_ev[s], h->stream));
}

float *fbuf(mc_handle h, DBuf &b, size_t count) {
  b.reserve(h->alloc, sizeof(float) * std::max<size_t>(count, 1));
  return b.as<float>();
}

// Krylov blocks are padded with zero columns to 4 (plain) or 8 (bf16 panels).
int block_align(mc_handle h) { return h->precision ? 8 : 4; }

// clamp as the oracle does: one block must fit, (p+1)(k+s) <= min(m, n), and
// the basis width (blocks padded to 4 columns) stays within kMaxKt.
void clamp_kp(mc_handle h, int s, int &k, int &p) {
  const int64_t lim = std::min(h->m, h->n);
  if (k + s > lim) k = std::max<int64_t>(1, lim - s);
  MC_REQUIRE(k + s <= lim, "k + s exceeds min(m, n)");
  const int kb = k + s;
  const int kbp = (int)round_up(kb, block_align(h));
  MC_REQUIRE(kbp <= kMaxKt, "k + s above the supported basis width (1024)");
  p = (int)std::max<int64_t>(0, std::min<int64_t>(p, lim / kb - 1));
  p = std::max(0, std::min(p, kMaxKt / kbp - 1));
}

// Brackets the launches issued in its scope with events when timing is on.
struct Scope {
  mc_handle h;
  int cat;
  double bytes, flops;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  Scope(mc_handle h_, int cat_, double bytes_ = 0, double flops_ = 0, cudaStream_t st_ = nullptr)
      : h(h_), cat(cat_), bytes(bytes_), flops(flops_), st(st_ ? st_ : h_->stream) {
    if (h->prof.on && (h->prof.mask >> cat & 1u)) {
      a = h->prof.get();
      MC_CUDA(cudaEventRecord(a, st));
    }
  }
  ~Scope() {
    if (a) {
      cudaEvent_t b = h->prof.get();
      cudaEventRecord(b, st);
      h->prof.pending.push_back({cat, a, b, bytes, flops});
    }
  }
};

// The main stream waits for a pending copy of Y into CSC order (before
// reading the CSC values, or writing Y or the copy).
void yc_ready(mc_handle h) {
  if (!h->yc_pending) return;
  MC_CUDA(cudaStreamWaitEvent(h->stream, h->ev_yc, 0));
  h->yc_pending = false;
}

// Copies the updated Y into CSC order on the side stream, after the work
// already on the main stream.
void mirror_async(mc_handle h) {
  yc_ready(h);
  if (h->single_stream) {
    Scope sc(h, MC_T_OTHER, 12.0 * h->nnz);
    mirror_values(h->stream, h->nnz, h->perm.as<int>(), h->y.as<float>(), h->yc.as<float>());
    return;
  }
  if (!h->side) {
    MC_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    MC_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    MC_CUDA(cudaEventCreateWithFlags(&h->ev_yc, cudaEventDisableTiming));
  }
  MC_CUDA(cudaEventRecord(h->ev_fork, h->stream));
  MC_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  {
    Scope sc(h, MC_T_OTHER, 12.0 * h->nnz, 0, h->side);
    mirror_values(h->side, h->nnz, h->perm.as<int>(), h->y.as<float>(), h->yc.as<float>());
  }
  MC_CUDA(cudaEventRecord(h->ev_yc, h->side));
  h->yc_pending = true;
}

double spmm_bytes(int64_t nnz, int64_t rows, int64_t rows_in, int K) {
  return 8.0 * nnz + 4.0 * (rows + 1) + 4.0 * (double)(rows_in + rows) * K;
}

// ---- SpMM launch-shape autotuner ----
// The first product of a shape class (direction, panel width, log2 of the
// row, input-row and entry counts) times every candidate launch shape twice
// with CUDA events on the handle's stream and keeps the fastest for the rest
// of the process.  The candidates differ only in launch shape, never in the
// order of any sum, so tuning cannot change a result.  MC_SPMM_TUNE=0 keeps
// the default shape; MC_SPMM_TUNE_LOG=1 prints the measurements to stderr.
// A shape class: direction, what the candidate launch shapes depend on (lane
// groups, default chunk, whether a half chunk is offered) and log2 of the
// rows, input rows and entries.  Panel widths with the same candidates share
// a class, so a served job whose k grows by a few columns, or a new job of a
// similar size, reuses the measured shape instead of timing the candidates
// again.
struct TuneKey {
  int trans, G, dc, wide, lr, lri, lnnz;
  bool operator<(const TuneKey &o) const {
    return std::tie(trans, G, dc, wide, lr, lri, lnnz) < std::tie(o.trans, o.G, o.dc, o.wide, o.lr, o.lri, o.lnnz);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, SpmmCfg> g_tune;

bool tune_enabled() {
  static const bool on = [] {
    const char *v = std::getenv("MC_SPMM_TUNE");
    return !(v && v[0] == '0');
  }();
  return on;
}
int ilog2(int64_t x) {
  int l = 0;
  while (x > 1) {
    x >>= 1;
    ++l;
  }
  return l;
}

// MC_SPMM_FORCE="u,threads,chunk" fixes the launch shape (tests compare
// shapes bit for bit; 0 fields keep their defaults).
const SpmmCfg *forced_cfg() {
  static const SpmmCfg cfg = [] {
    SpmmCfg c;
    c.u = -1;
    const char *v = std::getenv("MC_SPMM_FORCE");
    if (v) {
      int a = 0, b = 0, d = 0;
      if (std::sscanf(v, "%d,%d,%d", &a, &b, &d) == 3) c = SpmmCfg{a, b, d};
    }
    return c;
  }();
  return cfg.u >= 0 ? &cfg : nullptr;
}

template <class F>
SpmmCfg tuned_cfg(mc_handle h, int trans, int K, int64_t rows, int64_t rows_in, F &&launch) {
  if (const SpmmCfg *f = forced_cfg()) return *f;
  if (!tune_enabled()) return SpmmCfg{};
  const TuneKey key{trans, spmm_groups(K, rows_in), default_chunk(rows_in), K > 32 ? 1 : 0, ilog2(rows),
                    ilog2(rows_in), ilog2(std::max<int64_t>(h->nnz, 1))};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  const std::vector<SpmmCfg> cand = spmm_candidates(K, rows_in);
  if (cand.size() < 2) return SpmmCfg{};
  std::vector<cudaEvent_t> ev(2 * cand.size() * 2 + 1);
  for (auto &e : ev) MC_CUDA(cudaEventCreate(&e));
  int q = 0;
  MC_CUDA(cudaEventRecord(ev[q++], h->stream));
  for (int rep = 0; rep < 2; ++rep)
    for (const SpmmCfg &c : cand) {
      launch(c);
      MC_CUDA(cudaEventRecord(ev[q++], h->stream));
    }
  MC_CUDA(cudaEventSynchronize(ev[q - 1]));
  std::vector<float> best(cand.size(), 1e30f);
  for (int rep = 0, t = 1; rep < 2; ++rep)
    for (size_t i = 0; i < cand.size(); ++i, ++t) {
      float ms = 0.f;
      MC_CUDA(cudaEventElapsedTime(&ms, ev[t - 1], ev[t]));
      best[i] = std::min(best[i], ms);
    }
  for (auto &e : ev) cudaEventDestroy(e);
  size_t bi = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (best[i] < best[bi]) bi = i;
  static const bool log = [] {
    const char *v = std::getenv("MC_SPMM_TUNE_LOG");
    return v && v[0] == '1';
  }();
  if (log) {
    std::fprintf(stderr, "spmm tune trans=%d K=%d rows=%lld rows_in=%lld nnz=%lld:", trans, K, (long long)rows,
                 (long long)rows_in, (long long)h->nnz);
    for (size_t i = 0; i < cand.size(); ++i)
      std::fprintf(stderr, " [u%d t%d c%d %.1fus]", cand[i].u, cand[i].threads, cand[i].chunk, 1e3 * best[i]);
    std::fprintf(stderr, " -> %zu\n", bi);
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.emplace(key, cand[bi]);
  return cand[bi];
}

// ---- sparse products with the current iterate ----
void spmm_Y(mc_handle h, const float *X, int ld_x, int K, float *out, int ld_out) {
  fbuf(h, h->sp_part, (size_t)h->plan_r.nslot * K);
  auto run = [&](const SpmmCfg &c) {
    spmm(h->stream, h->plan_r, h->ci.as<int>(), h->y.as<float>(), h->n, X, ld_x, K, out, ld_out,
         h->sp_part.as<float>(), c);
  };
  const SpmmCfg cfg = tuned_cfg(h, 0, K, h->m, h->n, run);
  Scope sc(h, MC_T_SPMM, spmm_bytes(h->nnz, h->m, h->n, K), 2.0 * h->nnz * K);
  run(cfg);
}
// Products with bf16 panels (mixed-precision form); X has ld_x = K columns.
void spmm_Y_bf(mc_handle h, const void *X, int K, float *out, int ld_out) {
  fbuf(h, h->sp_part, (size_t)h->plan_r.nslot * K);
  Scope sc(h, MC_T_SPMM, 8.0 * h->nnz + 4.0 * (h->m + 1) + (2.0 * h->n + 4.0 * h->m) * K, 2.0 * h->nnz * K);
  spmm_bf16(h->stream, h->plan_r, h->ci.as<int>(), h->y.as<float>(), X, K, K, out, ld_out, h->sp_part.as<float>());
}
void spmm_Yt_bf(mc_handle h, const void *X, int K, float *out, int ld_out) {
  yc_ready(h);
  fbuf(h, h->sp_part, (size_t)h->plan_c.nslot * K);
  Scope sc(h, MC_T_SPMM_T, 8.0 * h->nnz + 4.0 * (h->n + 1) + (2.0 * h->m + 4.0 * h->n) * K, 2.0 * h->nnz * K);
  spmm_bf16(h->stream, h->plan_c, h->ri.as<int>(), h->yc.as<float>(), X, K, K, out, ld_out, h->sp_part.as<float>());
}
void *bf_panel(mc_handle h, DBuf &b, int64_t rows, int cols, const float *src, int ld_src) {
  b.reserve(h->alloc, 2 * (size_t)std::max<int64_t>(rows * cols, 1));
  Scope sc(h, MC_T_OTHER, 6.0 * rows * cols);
  to_bf16(h->stream, rows, cols, src, ld_src, b.p, cols);
  return b.p;
}

void spmm_Yt(mc_handle h, const float *X, int ld_x, int K, float *out, int ld_out) {
  yc_ready(h);
  fbuf(h, h->sp_part, (size_t)h->plan_c.nslot * K);
  auto run = [&](const SpmmCfg &c) {
    spmm(h->stream, h->plan_c, h->ri.as<int>(), h->yc.as<float>(), h->m, X, ld_x, K, out, ld_out,
         h->sp_part.as<float>(), c);
  };
  const SpmmCfg cfg = tuned_cfg(h, 1, K, h->n, h->m, run);
  Scope sc(h, MC_T_SPMM_T, spmm_bytes(h->nnz, h->n, h->m, K), 2.0 * h->nnz * K);
  run(cfg);
}

// Device flag of the handle that the tensor-core kernels raise when a bounded
// wait expires (checked after every Ritz eigensolve).
int *tc_err(mc_handle h) { return h->flags.p ? h->flags.as<int>() + 3 : nullptr; }

// The warp-specialised tensor-core X1^T X2 (through gemm_tn) takes this Gram
// (MC_TN_TC=0 and MC_GRAM_WS=0 keep the older tensor-core Gram above 64 columns).
bool tn_tc_covers(int64_t R, int K, const float *X, int ld) {
  static const bool on = [] {
    const char *v = std::getenv("MC_GRAM_WS");
    return !(v && v[0] == '0');
  }();
  const char *t = std::getenv("MC_TN_TC");
  return on && !(t && t[0] == '0') && K > 16 && gemm_tn_tc_supported(R, K, K, X, ld, X, ld);
}

// Gram X^T X: the tensor-core kernel (tcgen05, 3xTF32) for tc_min_k() <= K
// <= 256, SIMT otherwise; MC_GRAM_SIMT=1 selects SIMT everywhere.
bool use_tensor_gram() {
  static const bool on = [] {
    const char *v = std::getenv("MC_GRAM_SIMT");
    return !(v && v[0] == '1');
  }();
  return on;
}

int tc_min_k() {
  static const int v = [] {
    const char *e = std::getenv("MC_GRAM_TC_MIN_K");
    return e ? std::max(1, std::atoi(e)) : 65;
  }();
  return v;
}

void gram(mc_handle h, int64_t R, int K, const float *X, int ld, float *Gout, int ldg, const int *skip = nullptr) {
  Scope sc(h, MC_T_GRAM, 4.0 * R * K + 4.0 * K * K, 1.0 * R * K * (K + 1));
  if (!skip && use_tensor_gram() && K >= tc_min_k() && gram_tc_supported(K, ld, X) && !tn_tc_covers(R, K, X, ld)) {
    fbuf(h, h->tn_part, gram_tc_scratch_floats(R, K));
    gram_tc(h->stream, R, K, X, ld, Gout, ldg, h->tn_part.as<float>(), h->flags.as<int>() + 3);
    return;
  }
  fbuf(h, h->tn_part, gemm_tn_scratch_floats(R, K, K));
  gemm_tn(h->stream, R, K, K, X, ld, X, ld, Gout, ldg, true, h->tn_part.as<float>(), skip, tc_err(h));
}

// One CholeskyQR pass: out = X R^{-1} with X^T X + shift I = R^T R.
// set_skip: device flag set when this pass's Gram is within 1e-2 of I;
// skip_if: device flag that turns this pass into out = X (its Gram, factor
// and product are not computed).
void cholqr_pass(mc_handle h, int64_t R, int K, const float *X, int ldx, float *out, int ldo, float shift_rel,
                 const float *ref_diag = nullptr, int *set_skip = nullptr, const int *skip_if = nullptr) {
  float *G = fbuf(h, h->G, (size_t)K * K);
  gram(h, R, K, X, ldx, G, K, skip_if);
  float *Ri = fbuf(h, h->Rinv, (size_t)K * K);
  {
    // a column keeping less than 1e-5 of its norm through the projection is noise
    Scope sc(h, MC_T_SMALL);
    chol_inv(h->stream, K, G, K, shift_rel, ref_diag, 1e-10f, Ri, skip_if, set_skip);
  }
  Scope sc(h, MC_T_GEMM, 8.0 * R * K + 4.0 * K * K, 2.0 * R * K * K);
  gemm_nn(h->stream, R, K, K, X, ldx, Ri, K, nullptr, 1.0f, 0.0f, out, ldo, skip_if, tc_err(h));
}

// Orthonormal basis of range(X) (m x K, zero columns allowed) into out.
// Shifted CholeskyQR followed by CholeskyQR2 (three passes).  X is clobbered.
// For 16 < K <= 64 the third pass is decided on the device: when the second
// pass's Gram is within 1e-2 of I (the first pass already left the block
// orthonormal to that level) the second pass's result is final and the third
// only copies it, with no host round trip.
// ref_diag: optional column norms^2 of X before it was projected.
void orth_block(mc_handle h, int64_t R, int K, float *X, int ldx, float *out, int ldo,
                const float *ref_diag = nullptr) {
  float *tmp = fbuf(h, h->Tmp, (size_t)R * K);
  const bool dev_skip = K > 16 && K <= 64 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0 &&
                        h->flags.p != nullptr && h->flags.cap >= sizeof(int) * 8;
  int *flag = dev_skip ? h->flags.as<int>() + 4 : nullptr;
  cholqr_pass(h, R, K, X, ldx, tmp, K, 1e-6f, ref_diag);
  cholqr_pass(h, R, K, tmp, K, X, ldx, 0.0f, nullptr, flag);
  cholqr_pass(h, R, K, X, ldx, out, ldo, 0.0f, nullptr, nullptr, flag);
}

// X -= Qp (Qp^T X), twice (block classical Gram-Schmidt, reorthogonalised).
void project_out(mc_handle h, int64_t R, const float *Qp, int ldq, int cols, float *X, int K, int ldx) {
  if (cols <= 0) return;
  float *C = fbuf(h, h->C, (size_t)cols * K);
  fbuf(h, h->tn_part, gemm_tn_scratch_floats(R, cols, K));
  for (int rep = 0; rep < 2; ++rep) {
    {
      Scope sc(h, MC_T_GRAM, 4.0 * R * (cols + K), 2.0 * R * cols * K);
      gemm_tn(h->stream, R, cols, K, Qp, ldq, X, ldx, C, K, false, h->tn_part.as<float>(), nullptr, tc_err(h));
    }
    Scope sc(h, MC_T_GEMM, 4.0 * R * (cols + 2 * K), 2.0 * R * cols * K);
    gemm_nn(h->stream, R, cols, K, Qp, ldq, C, K, nullptr, -1.0f, 1.0f, X, ldx, nullptr, tc_err(h));
  }
}

// Omega (n x kbp, Kb real columns) for call id; optional warm-start columns.
void draw_omega(mc_handle h, int kb, int kbp, uint64_t seed, uint64_t call_id, const float *warm, int warm_ld,
                int warm_cols) {
  float *Om = fbuf(h, h->Om, (size_t)h->n * kbp);
  Scope sc(h, MC_T_OTHER, 4.0 * h->n * kbp);
  launch_omega(h->stream, h->n, kb, kbp, seed, call_id, 0, Om, nullptr);
  if (warm && warm_cols > 0)
    MC_CUDA(cudaMemcpy2DAsync(Om, sizeof(float) * kbp, warm, sizeof(float) * warm_ld, sizeof(float) * warm_cols, h->n,
                              cudaMemcpyDeviceToDevice, h->stream));
}

// Block-Krylov basis of Alg. 5 (steps 1-7) into h->Q (m x (p+1)*kbp).
// With the mixed-precision form the three panels that feed the Krylov
// products (Omega, A^T Q_{i-1} and Q_{i-1}) are read as bf16; sums stay
// float32 and the basis is orthonormalised in float32.
// The whole block step (norms, two projections against the first cols
// columns of Qp, the CholeskyQR passes) as one cooperative launch for narrow
// blocks; false when it does not apply (the caller runs the separate kernels).
// MC_ORTH_FUSED=0 turns it off.
bool orth_block_fused(mc_handle h, int64_t R, int K, float *X, int ldx, const float *Qp, int ldq, int cols, float *out,
                      int ldo) {
  static const bool on = [] {
    const char *v = std::getenv("MC_ORTH_FUSED");
    return !(v && v[0] == '0');
  }();
  if (!on || K > 32) return false;
  float *scr = fbuf(h, h->tn_part, orth_narrow_scratch_floats(R, K, cols));
  Scope sc(h, MC_T_GEMM, 4.0 * R * (2.0 * K + cols), 2.0 * R * K * (2.0 * cols + 1.5 * K));
  return orth_narrow(h->stream, R, K, X, ldx, Qp, ldq, cols, out, ldo, cols > 0, 1e-6f, 1e-10f, scr);
}

// Steps 3-7 of Alg. 5 for one block: out = an orthonormal basis of
// (I - Qp Qp^T) X (X clobbered), one cooperative launch for narrow blocks,
// else norms, two projections and three CholeskyQR passes as separate kernels
// (the one-launch form skips the third pass when the second leaves the block
// orthonormal to within 1e-2).
void orth_step(mc_handle h, int64_t R, int K, float *X, int ldx, const float *Qp, int ldq, int cols, float *out,
               int ldo) {
  if (orth_block_fused(h, R, K, X, ldx, Qp, ldq, cols, out, ldo)) return;
  if (cols <= 0) {
    orth_block(h, R, K, X, ldx, out, ldo);
    return;
  }
  float *ref = fbuf(h, h->lam, (size_t)K + colsumsq_scratch_floats(K));
  colsumsq(h->stream, R, K, X, ldx, ref, ref + K);
  project_out(h, R, Qp, ldq, cols, X, K, ldx);
  orth_block(h, R, K, X, ldx, out, ldo, ref);
}

void krylov_bki(mc_handle h, int kb, int p, uint64_t seed, uint64_t call_id, const float *warm, int warm_ld,
                int warm_cols) {
  const bool mixed = h->precision != 0;
  const int kbp = (int)round_up(kb, block_align(h));
  const int ktp = (p + 1) * kbp;
  draw_omega(h, kb, kbp, seed, call_id, warm, warm_ld, warm_cols);
  float *Q = fbuf(h, h->Q, (size_t)h->m * ktp);
  float *H = fbuf(h, h->H, (size_t)h->m * kbp);
  // Y^T Q_{i-1} of step i (float32 in both forms) is column block i-1 of
  // B^T = Y^T Q, so the Ritz step forms only the last block; the mixed form
  // rounds only the panel of the following Y (Y^T Q_{i-1}) product to bf16
  float *Bt = fbuf(h, h->Bt, (size_t)h->n * ktp);
  h->bt_ready = 0;
  if (mixed) spmm_Y_bf(h, bf_panel(h, h->Om_bf, h->n, kbp, h->Om.as<float>(), kbp), kbp, H, kbp);
  else spmm_Y(h, h->Om.as<float>(), kbp, kbp, H, kbp);  // H_0 = A Omega
  orth_step(h, h->m, kbp, H, kbp, nullptr, 0, 0, Q, ktp);
  for (int i = 1; i <= p; ++i) {
    float *Ti = Bt + (size_t)(i - 1) * kbp;
    spmm_Yt(h, Q + (size_t)(i - 1) * kbp, ktp, kbp, Ti, ktp);  // A^T Q_{i-1}
    if (mixed) spmm_Y_bf(h, bf_panel(h, h->T_bf, h->n, kbp, Ti, ktp), kbp, H, kbp);
    else spmm_Y(h, Ti, ktp, kbp, H, kbp);                     // A (A^T Q_{i-1})
    orth_step(h, h->m, kbp, H, kbp, Q, ktp, i * kbp, Q + (size_t)i * kbp, ktp);
  }
  h->Kq = ktp;
  h->q_real = (p + 1) * kb;
  h->bt_ready = p * kbp;
}

// Power-iteration basis of Alg. 4 (steps 1-7) into h->Q (m x kbp).
void power_pi(mc_handle h, int kb, int p, uint64_t seed, uint64_t call_id, const float *warm = nullptr,
              int warm_ld = 0, int warm_cols = 0) {
  const bool mixed = h->precision != 0;
  const int kbp = (int)round_up(kb, block_align(h));
  draw_omega(h, kb, kbp, seed, call_id, warm, warm_ld, warm_cols);
  float *Q = fbuf(h, h->Q, (size_t)h->m * kbp);
  float *H = fbuf(h, h->H, (size_t)h->m * kbp);
  float *T = fbuf(h, h->T, (size_t)h->n * kbp);
  if (mixed) spmm_Y_bf(h, bf_panel(h, h->Om_bf, h->n, kbp, h->Om.as<float>(), kbp), kbp, H, kbp);
  else spmm_Y(h, h->Om.as<float>(), kbp, kbp, H, kbp);  // Q = A Omega
  for (int i = 0; i < p; ++i) {
    orth_block(h, h->m, kbp, H, kbp, Q, kbp);      // lu(Q), an orthonormal basis of the same range
    if (mixed) {
      spmm_Yt_bf(h, bf_panel(h, h->Q_bf, h->m, kbp, Q, kbp), kbp, T, kbp);
      spmm_Y_bf(h, bf_panel(h, h->T_bf, h->n, kbp, T, kbp), kbp, H, kbp);
    } else {
      spmm_Yt(h, Q, kbp, kbp, T, kbp);
      spmm_Y(h, T, kbp, kbp, H, kbp);              // Q = A (A^T Q)
    }
  }
  orth_block(h, h->m, kbp, H, kbp, Q, kbp);        // eigSVD(Q): its U is an orthonormal basis (Lemma 2)
  h->Kq = kbp;
  h->q_real = kb;
}

// Basis of basic rSVD (Alg. 1, steps 1-7) into h->Q (m x kbp): Q = orth(A
// Omega), then p times G = orth(A^T Q), Q = orth(A G) -- an orthonormalisation
// after every product, the cost Alg. 4 halves.
void power_basic(mc_handle h, int kb, int p, uint64_t seed, uint64_t call_id) {
  const int kbp = (int)round_up(kb, 4);
  draw_omega(h, kb, kbp, seed, call_id, nullptr, 0, 0);
  float *Q = fbuf(h, h->Q, (size_t)h->m * kbp);
  float *H = fbuf(h, h->H, (size_t)h->m * kbp);
  float *T = fbuf(h, h->T, (size_t)h->n * kbp);
  float *G = fbuf(h, h->Bt, (size_t)h->n * kbp);
  spmm_Y(h, h->Om.as<float>(), kbp, kbp, H, kbp);
  orth_block(h, h->m, kbp, H, kbp, Q, kbp);        // Q = orth(A Omega)
  for (int i = 0; i < p; ++i) {
    spmm_Yt(h, Q, kbp, kbp, T, kbp);
    orth_block(h, h->n, kbp, T, kbp, G, kbp);      // G = orth(A^T Q)
    spmm_Y(h, G, kbp, kbp, H, kbp);
    orth_block(h, h->m, kbp, H, kbp, Q, kbp);      // Q = orth(A G)
  }
  h->Kq = kbp;
  h->q_real = kb;
}

// Steps 8-10 of Alg. 5 with basis Qb (m x Kq): B^T = A^T Qb, G = B B^T,
// top-kw eigenpairs (values to the host).
void ritz(mc_handle h, const float *Qb, int ldq, int Kq, int kw, bool fresh_krylov = false) {
  MC_REQUIRE(Kq <= kMaxKt, "basis wider than 1024");
  kw = std::min(kw, Kq);
  const int ready = fresh_krylov && ldq == Kq ? std::min(h->bt_ready, Kq) : 0;
  h->bt_ready = 0;
  float *Bt = ready > 0 ? h->Bt.as<float>() : fbuf(h, h->Bt, (size_t)h->n * Kq);
  spmm_Yt(h, Qb + ready, ldq, Kq - ready, Bt + ready, Kq);
  float *G = fbuf(h, h->G, (size_t)Kq * Kq);
  gram(h, h->n, Kq, Bt, Kq, G, Kq);
  float *lam = fbuf(h, h->lam, (size_t)Kq);
  float *W = fbuf(h, h->W, (size_t)Kq * kw);
  h->eig_work.reserve(h->alloc, eig_work_bytes(Kq, kw));
  {
    Scope sc(h, MC_T_EIG);
    eig_topk(h->stream, Kq, kw, G, Kq, lam, W, kw, h->eig_work.p);
  }
  h->h_lam.assign(kw, 0.f);
  MC_CUDA(cudaMemcpyAsync(h->h_lam.data(), lam, sizeof(float) * kw, cudaMemcpyDeviceToHost, h->stream));
  int werr = 0;
  MC_CUDA(cudaMemcpyAsync(&werr, h->flags.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  sync(h);
  if (werr) fail(MC_ETIMEOUT, "a bounded wait in the tensor-core Gram expired (code " + std::to_string(werr) + ")");
  h->Kq = Kq;
  h->kw = kw;
}

// Singular values from the Ritz eigenvalues: sigma = sqrt(lambda); values at
// or below the float32 noise floor K * eps * lambda_max are dropped (the
// rank-deficiency guard of eigSVD).
int ritz_sigmas(mc_handle h, int want, std::vector<double> &sig) {
  sig.clear();
  if (h->kw == 0) return 0;
  const double lmax = std::max<double>(h->h_lam[0], 0.0);
  const double floor_ = h->Kq * (double)std::numeric_limits<float>::epsilon() * lmax;
  for (int t = 0; t < std::min(want, h->kw); ++t) {
    const double l = h->h_lam[t];
    if (!(l > floor_) || l <= 0.0) break;
    sig.push_back(std::sqrt(l));
  }
  return (int)sig.size();
}

// U (m x ncols) = Qb W[:, :ncols] diag(su) and V (n x ncols) = B^T W[:, :ncols] diag(sv)
// with column counts padded to ldp (zeros).  Either output may be skipped.
void form_factors(mc_handle h, const float *Qb, int ldq, int ncols, const std::vector<double> &su,
                  const std::vector<double> &sv, float *U, float *V, int ldp) {
  const int Kq = h->Kq;
  float *Ws = fbuf(h, h->Wsel, (size_t)Kq * ldp);
  select_cols(h->stream, Kq, h->W.as<float>(), h->kw, ncols, ldp, Ws);
  std::vector<float> sc(2 * (size_t)ldp, 0.f);
  for (int j = 0; j < ncols; ++j) {
    sc[j] = (float)su[j];
    sc[ldp + j] = (float)sv[j];
  }
  float *dsc = fbuf(h, h->scale, 2 * (size_t)ldp);
  stage_copy(h, dsc, sc.data(), sc.size());
  if (U) {
    Scope sc(h, MC_T_GEMM, 4.0 * h->m * (Kq + ldp), 2.0 * h->m * Kq * ldp);
    gemm_nn(h->stream, h->m, Kq, ldp, Qb, ldq, Ws, ldp, dsc, 1.0f, 0.0f, U, ldp, nullptr, tc_err(h));
  }
  if (V) {
    Scope sc(h, MC_T_GEMM, 4.0 * h->n * (Kq + ldp), 2.0 * h->n * Kq * ldp);
    gemm_nn(h->stream, h->n, Kq, ldp, h->Bt.as<float>(), Kq, Ws, ldp, dsc + ldp, 1.0f, 0.0f, V, ldp, nullptr,
            tc_err(h));
  }
}

// Full rSVD into user buffers.
// algo: 0 rSVD-PI (Alg. 4), 1 rSVD-BKI (Alg. 5), 2 basic rSVD (Alg. 1).
mc_status do_rsvd(mc_handle h, int algo, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U, float *S,
                  float *V, int *k_out) {
  MC_REQUIRE(k >= 1 && s >= 0, "k must be >= 1 and s >= 0");
  const bool bki = algo == 1;
  if (bki) {
    clamp_kp(h, s, k, p);
  } else {
    // one block of k + s columns whatever p (Alg. 1 and 4 keep the width)
    int p1 = 0;
    clamp_kp(h, s, k, p1);
    p = std::max(p, 0);
  }
  const int kb = k + s;
  if (bki) krylov_bki(h, kb, p, seed, call_id, nullptr, 0, 0);
  else if (algo == 0) power_pi(h, kb, p, seed, call_id);
  else power_basic(h, kb, p, seed, call_id);
  ritz(h, h->Q.as<float>(), h->Kq, h->Kq, k, bki);
  std::vector<double> sig;
  const int kk = ritz_sigmas(h, k, sig);
  const int ldp = (int)round_up(std::max(kk, 1), 4);
  std::vector<double> ones(kk, 1.0), inv(kk);
  for (int j = 0; j < kk; ++j) inv[j] = 1.0 / sig[j];
  float *dU = fbuf(h, h->U, (size_t)h->m * ldp);
  float *dV = fbuf(h, h->V, (size_t)h->n * ldp);
  if (kk > 0) form_factors(h, h->Q.as<float>(), h->Kq, kk, ones, inv, U ? dU : nullptr, V ? dV : nullptr, ldp);
  copy_out_2d(h->stream, U, kk, dU, ldp, h->m);
  copy_out_2d(h->stream, V, kk, dV, ldp, h->n);
  if (S && kk > 0) {
    std::vector<float> hs(kk);
    for (int j = 0; j < kk; ++j) hs[j] = (float)sig[j];
    MC_CUDA(cudaMemcpyAsync(S, hs.data(), sizeof(float) * kk, cudaMemcpyDefault, h->stream));
    sync(h);
  }
  sync(h);
  if (k_out) *k_out = kk;
  return MC_OK;
}

// ---------------------------------------------------------------- SVT ------
double sumsq_values(mc_handle h, const float *v, int64_t count) {
  h->dsum.reserve(h->alloc, sizeof(double) * 1032);
  double *d = h->dsum.as<double>();
  sumsq_floats(h->stream, v, count, d + 8, d);
  double out = 0;
  MC_CUDA(cudaMemcpyAsync(&out, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  sync(h);
  return out;
}

// ||P_Phi(M)||_2 by power iteration on A^T A started from Omega column 0 of
// call 0 (float32 products, stopped at relative change 1e-7 of lambda).
double spectral_norm(mc_handle h, uint64_t seed) {
  float *v = fbuf(h, h->T, (size_t)h->n * 4);
  float *u = fbuf(h, h->H, (size_t)h->m * 4);
  float *w = fbuf(h, h->Tmp, (size_t)h->n * 4);
  launch_omega(h->stream, h->n, 1, 4, seed, 0, 0, v, nullptr);
  double nv = std::sqrt(sumsq_values(h, v, h->n * 4));
  if (nv == 0) return 0;
  scale_values(h->stream, h->n * 4, v, (float)(1.0 / nv), v);
  double lam_old = 0, lam = 0;
  for (int it = 0; it < 1000; ++it) {
    spmm_Y(h, v, 4, 4, u, 4);
    spmm_Yt(h, u, 4, 4, w, 4);
    lam = std::sqrt(sumsq_values(h, w, h->n * 4));
    if (lam == 0) return 0;
    scale_values(h->stream, h->n * 4, w, (float)(1.0 / lam), v);
    if (std::fabs(lam - lam_old) <= 1e-7 * lam) break;
    lam_old = lam;
  }
  return std::sqrt(lam);
}

void svt_initialise(mc_handle h, const mc_params *prm) {
  h->prm = *prm;
  const mc_params &P = h->prm;
  MC_REQUIRE(P.delta > 0 && P.eps > 0 && P.l >= 1 && P.s >= 0 && P.i_max >= 1, "invalid SVT parameters");
  MC_REQUIRE(P.recycle >= 0 && P.recycle <= 3, "recycle must be 0..3");
  MC_REQUIRE(P.precision == 0 || P.precision == 1, "precision must be 0 (float32) or 1 (bf16 panels)");
  MC_REQUIRE(P.inner == 0 || P.inner == 1, "inner must be 0 (rSVD-BKI) or 1 (rSVD-PI)");
  h->precision = P.precision;
  h->tau = P.tau > 0 ? P.tau : 5.0 * std::sqrt((double)h->m * (double)h->n);
  // Y currently holds P_Phi(M) only if no rSVD/SVT changed it; start from M.
  yc_ready(h);
  copy_in(h->stream, h->y.p, h->mval.p, sizeof(float) * h->nnz);
  mirror_values(h->stream, h->nnz, h->perm.as<int>(), h->y.as<float>(), h->yc.as<float>());
  h->normF = std::sqrt(sumsq_values(h, h->mval.as<float>(), h->nnz));
  h->norm2 = spectral_norm(h, P.seed);
  h->c = std::ceil(h->tau / (P.delta * h->norm2));
  scale_values(h->stream, h->nnz, h->mval.as<float>(), (float)(h->c * P.delta), h->y.as<float>());
  mirror_values(h->stream, h->nnz, h->perm.as<int>(), h->y.as<float>(), h->yc.as<float>());
  h->it = 0;
  h->r = 0;
  h->q = 0;
  h->p = P.p0;
  h->streak = 0;
  h->prev_err = std::numeric_limits<double>::infinity();
  h->call_id = 1;
  h->basis = 0;
  h->ub_k = 0;
  h->vb_k = 0;
  h->r_cur = 0;
  h->svt_init = true;
  sync(h);
}

// One SVD call of the repeat loop.  Returns the singular values (descending)
// in sig; leaves W/Bt/Kq ready for form_factors with basis pointer *Qb.
void svt_svd(mc_handle h, int kk, int pp, bool fresh, std::vector<double> &sig, const float **Qb, int *ldq) {
  const mc_params &P = h->prm;
  if (fresh) {
    const float *warm = nullptr;
    int wcols = 0;
    if (P.recycle == 3 && h->vb_k > 0 && h->r > 0) {
      warm = h->Vb.as<float>();
      wcols = std::min(std::min(h->r, kk + P.s), h->vb_k);
    }
    if (P.inner == 1) power_pi(h, kk + P.s, pp, P.seed, h->call_id, warm, h->vb_ld, wcols);
    else krylov_bki(h, kk + P.s, pp, P.seed, h->call_id, warm, h->vb_ld, wcols);
    h->call_id += 1;
    ritz(h, h->Q.as<float>(), h->Kq, h->Kq, kk, P.inner != 1);
    *Qb = h->Q.as<float>();
    *ldq = h->Kq;
    if (P.recycle == 1) h->basis = 1;
  } else if (P.recycle == 1) {
    ritz(h, h->Q.as<float>(), h->Kq, h->Kq, kk);  // strategy 1: restart at step 8 with the stored Q
    *Qb = h->Q.as<float>();
    *ldq = h->Kq;
  } else {
    // strategy 2: B = U^T Y, eigSVD(B^T), U <- U W (all k_prev triplets)
    ritz(h, h->Ub.as<float>(), h->ub_ld, h->ub_ld, h->ub_k);
    *Qb = h->Ub.as<float>();
    *ldq = h->ub_ld;
  }
  ritz_sigmas(h, h->kw, sig);
}

mc_status svt_step(mc_handle h, mc_iter_info *out) {
  const mc_params &P = h->prm;
  h->it += 1;
  const int it = h->it;
  int k = h->r + 1;
  bool force_fresh = false, used_recycle = false;
  int nsvd = 0, kk = 0;
  std::vector<double> sig;
  const float *Qb = nullptr;
  int ldq = 0;
  const int64_t lim = std::min(h->m, h->n);
  int k_cap = (int)(lim - P.s);
  if (P.k_max > 0) k_cap = std::min(k_cap, P.k_max);
  for (;;) {
    kk = std::min(k, std::max(1, k_cap));
    int pp = h->p;
    if (P.inner == 1) {
      int p1 = 0;  // rSVD-PI keeps one block of k + s columns whatever p
      clamp_kp(h, P.s, kk, p1);
    } else {
      clamp_kp(h, P.s, kk, pp);
    }
    bool width_ok = false;
    if (P.recycle == 1) width_ok = h->basis == 1 && h->q_real >= kk;
    if (P.recycle == 2) width_ok = h->basis == 2 && h->ub_k >= kk;
    const bool fresh = P.recycle == 0 || P.recycle == 3 || it < P.i_reuse || h->q == P.q_reuse || !width_ok ||
                       force_fresh;
    svt_svd(h, kk, pp, fresh, sig, &Qb, &ldq);
    if (fresh) {
      h->q = 0;
    } else {
      h->q += 1;
      used_recycle = true;
    }
    nsvd += 1;
    k += P.l;
    const int got = (int)sig.size();
    if (P.recycle == 2) {
      // the basis for the next recycled call is this call's U (all triplets)
      const int ldp = (int)round_up(std::max(got, 1), 4);
      std::vector<double> ones(got, 1.0), z(got, 0.0);
      float *Unew = fbuf(h, h->U, (size_t)h->m * ldp);
      if (got > 0) form_factors(h, Qb, ldq, got, ones, z, Unew, nullptr, ldp);
      std::swap(h->U, h->Ub);
      h->ub_k = got;
      h->ub_ld = ldp;
      h->basis = 2;
      Qb = nullptr;
    }
    const double last = got > 0 ? sig[got - 1] : 0.0;
    if (got == 0 || last <= h->tau) break;
    if (kk >= lim - P.s || (P.k_max > 0 && kk >= P.k_max)) break;
    if (!fresh) force_fresh = true;
  }
  const int got = (int)sig.size();
  int r = 0;
  while (r < got && sig[r] > h->tau) ++r;
  // shrunk factors: Us = U(:, 1:r) diag(sigma - tau), V_r = B^T W S^-1
  const int ldp = (int)round_up(std::max(r, 1), 4);
  std::vector<double> su(r), sv(r);
  for (int j = 0; j < r; ++j) {
    su[j] = sig[j] - h->tau;
    sv[j] = 1.0 / sig[j];
  }
  float *Us = fbuf(h, h->U, (size_t)h->m * ldp);
  float *Vr = fbuf(h, h->V, (size_t)h->n * ldp);
  if (r > 0) {
    if (P.recycle == 2) {
      // U is the stored basis already rotated: Us = Ub(:, 1:r) diag(sigma - tau)
      std::vector<double> id(r, 0.0);
      // Ub holds U; B^T for V is in h->Bt with W of the last ritz (basis = old Ub)
      // V_r from the last ritz call; Us by scaling the first r columns of Ub.
      form_factors(h, nullptr, 0, r, su, sv, nullptr, Vr, ldp);
      float *Ws = fbuf(h, h->Wsel, (size_t)h->ub_ld * ldp);
      std::vector<float> eye((size_t)h->ub_ld * ldp, 0.f);
      for (int j = 0; j < r; ++j) eye[(size_t)j * ldp + j] = (float)su[j];
      stage_copy(h, Ws, eye.data(), eye.size());
      gemm_nn(h->stream, h->m, h->ub_ld, ldp, h->Ub.as<float>(), h->ub_ld, Ws, ldp, nullptr, 1.0f, 0.0f, Us, ldp,
              nullptr, tc_err(h));
    } else {
      form_factors(h, Qb, ldq, r, su, sv, Us, Vr, ldp);
    }
  } else {
    MC_CUDA(cudaMemsetAsync(Us, 0, sizeof(float) * h->m * ldp, h->stream));
    MC_CUDA(cudaMemsetAsync(Vr, 0, sizeof(float) * h->n * ldp, h->stream));
  }
  h->r = r;
  h->r_cur = r;
  h->us_ld = ldp;
  h->sig = sig;
  // warm-start block for recycle = 3: the previous V (first r columns suffice)
  if (P.recycle == 3) {
    float *Vb = fbuf(h, h->Vb, (size_t)h->n * ldp);
    MC_CUDA(cudaMemcpyAsync(Vb, Vr, sizeof(float) * h->n * ldp, cudaMemcpyDeviceToDevice, h->stream));
    h->vb_k = r;
    h->vb_ld = ldp;
  }
  // fused SDDMM + residual + update over Phi, then mirror Y into the CSC copy
  double *sq = reinterpret_cast<double *>(fbuf(h, h->seg_sq, 2 * (size_t)sddmm_partials() + 16));
  int nsq = 0;
  yc_ready(h);  // the previous copy into CSC order has read Y
  {
    Scope sc(h, MC_T_SDDMM, 20.0 * h->nnz + 4.0 * (double)(h->m + h->n) * ldp, 2.0 * h->nnz * r);
    nsq = sddmm_update(h->stream, h->nnz, h->rix.as<int>(), h->ci.as<int>(), h->mval.as<float>(), h->y.as<float>(),
                       Us, ldp, Vr, ldp, r, (float)P.delta, 1, sq, nullptr);
  }
  h->dsum.reserve(h->alloc, sizeof(double) * 1032);
  mirror_async(h);  // Y -> CSC order, overlapping what follows
  {
    Scope sc(h, MC_T_OTHER, 0);
    sum_doubles(h->stream, sq, nsq, h->dsum.as<double>());
  }
  double ssq = 0;
  MC_CUDA(cudaMemcpyAsync(&ssq, h->dsum.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  sync(h);
  const double err = std::sqrt(ssq) / h->normF;
  h->last_err = err;
  if (!std::isfinite(err)) fail(MC_EINTERNAL, "non-finite residual on Phi at iteration " + std::to_string(it));
  const bool conv = err < P.eps;
  if (!conv) {
    if (err > h->prev_err) {
      h->p = std::min(h->p + 1, P.p_max);
      h->streak = 0;
    } else if (err < h->prev_err) {
      h->streak += 1;
      if (h->streak == 10) {
        h->p = std::max(h->p - 1, P.p_min);
        h->streak = 0;
      }
    } else {
      h->streak = 0;
    }
    h->prev_err = err;
  }
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->i = it;
    out->k = kk;
    out->r = r;
    out->p = h->p;
    out->nsvd = nsvd;
    out->recycled = used_recycle ? 1 : 0;
    out->converged = conv ? 1 : 0;
    out->err = err;
    out->sigma_last = got > 0 ? sig[got - 1] : 0.0;
    out->sigma_max = got > 0 ? sig[0] : 0.0;
    out->c = h->c;
    out->norm2 = h->norm2;
  }
  return MC_OK;
}

template <class F>
mc_status guarded(F &&f) {
  try {
    return f();
  } catch (const Err &e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return MC_ENOMEM;
  } catch (const std::exception &e) {
    set_error(e.what());
    return MC_EINTERNAL;
  }
}

}  // namespace

// ====================================================================== ABI ==
extern "C" {

void mc_params_default(mc_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tau = 0.0;
  p->delta = 1.2;
  p->eps = 1e-4;
  p->l = 5;
  p->s = 10;
  p->p0 = 3;
  p->p_min = 3;
  p->p_max = 20;
  p->i_max = 1000;
  p->i_reuse = 50;
  p->q_reuse = 10;
  p->recycle = 1;
  p->k_max = 0;
  p->precision = 0;
  p->inner = 0;
  p->seed = 0;
}

const char *mc_last_error(void) { return g_last_error.c_str(); }

int64_t mc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *mc_status_str(mc_status s) {
  switch (s) {
    case MC_OK: return "MC_OK";
    case MC_EINVAL: return "MC_EINVAL";
    case MC_ENOMEM: return "MC_ENOMEM";
    case MC_ECUDA: return "MC_ECUDA";
    case MC_ENOTCONVERGED: return "MC_ENOTCONVERGED";
    case MC_EBUSY: return "MC_EBUSY";
    case MC_PENDING: return "MC_PENDING";
    case MC_ETIMEOUT: return "MC_ETIMEOUT";
    case MC_ECANCELLED: return "MC_ECANCELLED";
    case MC_EINTERNAL: return "MC_EINTERNAL";
  }
  return "MC_UNKNOWN";
}

mc_status mc_create(mc_handle *out, int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                    const float *val, void *stream, const mc_allocator *alloc) {
  if (!out) return MC_EINVAL;
  *out = nullptr;
  std::unique_ptr<mc_handle_s> h(new (std::nothrow) mc_handle_s());
  if (!h) return MC_ENOMEM;
  mc_status st = guarded([&]() -> mc_status {
    MC_REQUIRE(m >= 1 && n >= 1, "m and n must be >= 1");
    MC_REQUIRE(m < (int64_t(1) << 31) && n < (int64_t(1) << 31), "m and n must be < 2^31");
    MC_REQUIRE(nnz >= 0 && nnz < (int64_t(1) << 31), "nnz must be in [0, 2^31)");
    MC_REQUIRE(row_ptr && (nnz == 0 || (col && val)), "null input array");
    if (alloc) {
      MC_REQUIRE(alloc->alloc && alloc->free, "allocator hook needs alloc and free");
      h->alloc.hook = *alloc;
      h->alloc.has_hook = true;
    }
    if (stream) {
      h->stream = static_cast<cudaStream_t>(stream);
    } else {
      MC_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
      h->own_stream = true;
    }
    h->alloc.stream = h->stream;
    h->m = m;
    h->n = n;
    h->nnz = nnz;
    cudaStream_t s = h->stream;
    // row_ptr (int64) -> int32 with checks
    DBuf rp64;
    BufGuard g_rp64(h->alloc, {&rp64});
    rp64.reserve(h->alloc, sizeof(int64_t) * (m + 1));
    copy_in(s, rp64.p, row_ptr, sizeof(int64_t) * (m + 1));
    h->rp.reserve(h->alloc, sizeof(int) * (m + 1));
    h->flags.reserve(h->alloc, sizeof(int) * 8);
    MC_CUDA(cudaMemsetAsync(h->flags.p, 0, sizeof(int) * 8, s));
    convert_rowptr(s, m, nnz, rp64.as<int64_t>(), h->rp.as<int>(), h->flags.as<int>());
    int fl[4] = {0, 0, 0, 0};
    MC_CUDA(cudaMemcpyAsync(fl, h->flags.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    rp64.release(h->alloc);
    MC_REQUIRE(fl[0] == 0, "row_ptr is not a valid CSR row pointer (must start at 0, be non-decreasing, end at nnz)");
    h->ci.reserve(h->alloc, sizeof(int) * std::max<int64_t>(nnz, 1));
    h->mval.reserve(h->alloc, sizeof(float) * std::max<int64_t>(nnz, 1));
    h->y.reserve(h->alloc, sizeof(float) * std::max<int64_t>(nnz, 1));
    copy_in(s, h->ci.p, col, sizeof(int) * nnz);
    copy_in(s, h->mval.p, val, sizeof(float) * nnz);
    validate_csr(s, m, n, h->rp.as<int>(), h->ci.as<int>(), h->mval.as<float>(), h->flags.as<int>());
    MC_CUDA(cudaMemcpyAsync(fl, h->flags.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    MC_REQUIRE(!(fl[1] & 1), "column index out of range");
    MC_REQUIRE(!(fl[1] & 2), "columns must be strictly increasing within each row (sorted, no duplicates)");
    MC_REQUIRE(fl[2] == 0, "values must be finite");
    copy_in(s, h->y.p, h->mval.p, sizeof(float) * nnz);
    h->rix.reserve(h->alloc, sizeof(int) * std::max<int64_t>(nnz, 1));
    expand_rows(s, m, h->rp.as<int>(), h->rix.as<int>());
    // CSC copy
    h->cp.reserve(h->alloc, sizeof(int) * (n + 1));
    h->ri.reserve(h->alloc, sizeof(int) * std::max<int64_t>(nnz, 1));
    h->perm.reserve(h->alloc, sizeof(int) * std::max<int64_t>(nnz, 1));
    h->yc.reserve(h->alloc, sizeof(float) * std::max<int64_t>(nnz, 1));
    DBuf tmp;
    BufGuard g_tmp(h->alloc, {&tmp});
    tmp.reserve(h->alloc, csc_tmp_bytes(m, n));
    build_csc(s, m, n, nnz, h->rp.as<int>(), h->ci.as<int>(), h->cp.as<int>(), h->ri.as<int>(), h->perm.as<int>(),
              tmp.p);
    MC_CUDA(cudaStreamSynchronize(s));
    tmp.release(h->alloc);
    mirror_values(s, nnz, h->perm.as<int>(), h->y.as<float>(), h->yc.as<float>());
    plan_segments(s, h->alloc, m, h->rp.as<int>(), h->plan_r);
    plan_segments(s, h->alloc, n, h->cp.as<int>(), h->plan_c);
    MC_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
  });
  if (st != MC_OK) {
    mc_destroy(h.release());
    return st;
  }
  *out = h.release();
  return MC_OK;
}

mc_status mc_create_coo(mc_handle *out, int64_t m, int64_t n, int64_t nnz, const int64_t *rows, const int32_t *cols,
                        const float *vals, void *stream, const mc_allocator *alloc) {
  if (!out) return MC_EINVAL;
  *out = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  bool own = false;
  Alloc a;
  DBuf r_d, c_d, v_d, rp, ci, va, fl;
  mc_status res = guarded([&]() -> mc_status {
    MC_REQUIRE(m >= 1 && n >= 1, "m and n must be >= 1");
    MC_REQUIRE(m < (int64_t(1) << 31) && n < (int64_t(1) << 31), "m and n must be < 2^31");
    MC_REQUIRE(nnz >= 0 && nnz < (int64_t(1) << 31), "nnz must be in [0, 2^31)");
    MC_REQUIRE(nnz == 0 || (rows && cols && vals), "null input array");
    if (!st) {
      MC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      own = true;
    }
    if (alloc) {
      MC_REQUIRE(alloc->alloc && alloc->free, "allocator hook needs alloc and free");
      a.hook = *alloc;
      a.has_hook = true;
    }
    a.stream = st;
    const size_t nz = (size_t)std::max<int64_t>(nnz, 1);
    r_d.reserve(a, sizeof(int64_t) * nz);
    c_d.reserve(a, sizeof(int) * nz);
    v_d.reserve(a, sizeof(float) * nz);
    rp.reserve(a, sizeof(int64_t) * (m + 1));
    ci.reserve(a, sizeof(int) * nz);
    va.reserve(a, sizeof(float) * nz);
    fl.reserve(a, sizeof(int) * 4);
    MC_CUDA(cudaMemsetAsync(fl.p, 0, sizeof(int) * 4, st));
    copy_in(st, r_d.p, rows, sizeof(int64_t) * nnz);
    copy_in(st, c_d.p, cols, sizeof(int) * nnz);
    copy_in(st, v_d.p, vals, sizeof(float) * nnz);
    coo_to_csr(st, a, m, n, nnz, r_d.as<int64_t>(), c_d.as<int>(), v_d.as<float>(), rp.as<int64_t>(), ci.as<int>(),
               va.as<float>(), fl.as<int>());
    int h_fl[4] = {0, 0, 0, 0};
    MC_CUDA(cudaMemcpyAsync(h_fl, fl.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    MC_CUDA(cudaStreamSynchronize(st));
    MC_REQUIRE(!(h_fl[1] & 1), "row or column index out of range");
    MC_REQUIRE(!(h_fl[1] & 2), "repeated (row, column) entry");
    MC_REQUIRE(h_fl[2] == 0, "values must be finite");
    return MC_OK;
  });
  if (res == MC_OK)
    res = mc_create(out, m, n, nnz, rp.as<int64_t>(), ci.as<int>(), va.as<float>(), own ? nullptr : stream, alloc);
  if (st) cudaStreamSynchronize(st);
  for (DBuf *b : {&r_d, &c_d, &v_d, &rp, &ci, &va, &fl}) b->release(a);
  if (own && st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  return res;
}

void mc_destroy(mc_handle h) {
  if (!h) return;
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->stream) cudaStreamSynchronize(h->stream);
  Alloc &a = h->alloc;
  for (DBuf *b : {&h->Om_bf, &h->Q_bf, &h->T_bf}) b->release(a);
  for (DBuf *b : {&h->rp, &h->ci, &h->mval, &h->y, &h->rix, &h->cp, &h->ri, &h->perm, &h->yc, &h->Om, &h->Q, &h->H, &h->Tmp,
                  &h->T, &h->Bt, &h->G, &h->C, &h->Rinv, &h->lam, &h->W, &h->Wsel, &h->scale, &h->U, &h->V, &h->Ub,
                  &h->Vb, &h->seg_sq, &h->dsum, &h->tn_part, &h->sp_part, &h->eig_work, &h->flags})
    b->release(a);
  for (SegPlan *pl : {&h->plan_r, &h->plan_c})
    for (DBuf *b : {&pl->seg, &pl->split_row, &pl->split_slot})
      b->release(a);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int q = 0; q < 2; ++q) {
    if (h->stage_ev[q]) cudaEventDestroy(h->stage_ev[q]);
    if (h->h_stage[q]) cudaFreeHost(h->h_stage[q]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_yc) cudaEventDestroy(h->ev_yc);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

mc_status mc_join(mc_handle h) {
  if (!h) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    yc_ready(h);
    return MC_OK;
  });
}

mc_status mc_set_values(mc_handle h, const float *val) {
  if (!h || (!val && h->nnz > 0)) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    yc_ready(h);
    copy_in(h->stream, h->y.p, val, sizeof(float) * h->nnz);
    mirror_values(h->stream, h->nnz, h->perm.as<int>(), h->y.as<float>(), h->yc.as<float>());
    sync(h);
    return MC_OK;
  });
}

mc_status mc_get_values(mc_handle h, float *val) {
  if (!h || (!val && h->nnz > 0)) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    MC_CUDA(cudaMemcpyAsync(val, h->y.p, sizeof(float) * h->nnz, cudaMemcpyDefault, h->stream));
    sync(h);
    return MC_OK;
  });
}

mc_status mc_rsvd_bki(mc_handle h, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U, float *S, float *V,
                      int *k_out) {
  if (!h) return MC_EINVAL;
  return guarded([&]() { return do_rsvd(h, 1, k, s, p, seed, call_id, U, S, V, k_out); });
}

mc_status mc_rsvd_pi(mc_handle h, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U, float *S, float *V,
                     int *k_out) {
  if (!h) return MC_EINVAL;
  return guarded([&]() { return do_rsvd(h, 0, k, s, p, seed, call_id, U, S, V, k_out); });
}

mc_status mc_rsvd_basic(mc_handle h, int k, int s, int p, uint64_t seed, uint64_t call_id, float *U, float *S,
                        float *V, int *k_out) {
  if (!h) return MC_EINVAL;
  return guarded([&]() { return do_rsvd(h, 2, k, s, p, seed, call_id, U, S, V, k_out); });
}

mc_status mc_set_precision(mc_handle h, int precision) {
  if (!h || (precision != 0 && precision != 1)) return MC_EINVAL;
  h->precision = precision;
  return MC_OK;
}

mc_status mc_svt_reset(mc_handle h) {
  if (!h) return MC_EINVAL;
  h->svt_init = false;
  return MC_OK;
}

mc_status mc_svt_step(mc_handle h, const mc_params *params, mc_iter_info *out) {
  if (!h) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    if (!h->svt_init) {
      MC_REQUIRE(params != nullptr, "the first mc_svt_step needs parameters");
      svt_initialise(h, params);
    }
    return svt_step(h, out);
  });
}

mc_status mc_svt_solve(mc_handle h, const mc_params *params, mc_iter_info *out) {
  if (!h || !params) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    svt_initialise(h, params);
    mc_iter_info info{};
    for (int i = 0; i < params->i_max; ++i) {
      svt_step(h, &info);
      if (info.converged) break;
    }
    if (out) *out = info;
    return info.converged ? MC_OK : MC_ENOTCONVERGED;
  });
}

mc_status mc_svt_factors(mc_handle h, int max_r, float *Us, float *V, float *sigma, int *r_out) {
  if (!h) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    MC_REQUIRE(h->svt_init, "no SVT estimate yet");
    const int r = h->r_cur;
    if (r_out) *r_out = r;
    MC_REQUIRE(r <= max_r || (!Us && !V && !sigma), "r exceeds max_r");
    copy_out_2d(h->stream, Us, r, h->U.as<float>(), h->us_ld, h->m);
    copy_out_2d(h->stream, V, r, h->V.as<float>(), h->us_ld, h->n);
    if (sigma && r > 0) {
      std::vector<float> s(r);
      for (int j = 0; j < r; ++j) s[j] = (float)h->sig[j];
      MC_CUDA(cudaMemcpyAsync(sigma, s.data(), sizeof(float) * r, cudaMemcpyDefault, h->stream));
      sync(h);
    }
    sync(h);
    return MC_OK;
  });
}

mc_status mc_svt_sample(mc_handle h, int64_t count, const int64_t *rows, const int64_t *cols, float *out) {
  if (!h || count < 0) return MC_EINVAL;
  if (count == 0) return MC_OK;
  return guarded([&]() -> mc_status {
    MC_REQUIRE(h->svt_init, "no SVT estimate yet");
    MC_REQUIRE(rows && cols && out, "null argument");
    DBuf dr, dc, dout;
    BufGuard g_bufs(h->alloc, {&dr, &dc, &dout});
    dr.reserve(h->alloc, sizeof(int64_t) * count);
    dc.reserve(h->alloc, sizeof(int64_t) * count);
    dout.reserve(h->alloc, sizeof(float) * count);
    copy_in(h->stream, dr.p, rows, sizeof(int64_t) * count);
    copy_in(h->stream, dc.p, cols, sizeof(int64_t) * count);
    sample_lowrank(h->stream, count, dr.as<int64_t>(), dc.as<int64_t>(), h->U.as<float>(), h->us_ld, h->V.as<float>(),
                   h->us_ld, h->r_cur, dout.as<float>());
    MC_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(float) * count, cudaMemcpyDefault, h->stream));
    sync(h);
    dr.release(h->alloc);
    dc.release(h->alloc);
    dout.release(h->alloc);
    sync(h);
    return MC_OK;
  });
}

mc_status mc_panel_gram(int64_t R, int K1, int K2, const float *X1, const float *X2, float *C, int tensor_cores) {
  if (R < 1 || K1 < 1 || K2 < 1 || !X1 || !X2 || !C) return MC_EINVAL;
  const int k1p = (int)round_up(K1, 4), k2p = (int)round_up(K2, 4);
  const bool same = X1 == X2 && K1 == K2;  // a Gram: one staged panel serves both operands
  if (tensor_cores && !gemm_tn_tc_supported(R, K1, K2, reinterpret_cast<const void *>(256), k1p,
                                            reinterpret_cast<const void *>(same ? 256 : 512), k2p))
    return MC_EINVAL;
  return guarded([&]() -> mc_status {
    DBuf d1, d2, dc, dp, de;
    Alloc a;
    BufGuard g(a, {&d1, &d2, &dc, &dp, &de});
    d1.reserve(a, sizeof(float) * R * k1p);
    d2.reserve(a, sizeof(float) * R * k2p);
    dc.reserve(a, sizeof(float) * K1 * K2);
    dp.reserve(a, sizeof(float) * gemm_tn_scratch_floats(R, K1, K2));
    de.reserve(a, sizeof(int));
    MC_CUDA(cudaMemset(de.p, 0, sizeof(int)));
    MC_CUDA(cudaMemset(d1.p, 0, sizeof(float) * R * k1p));
    MC_CUDA(cudaMemset(d2.p, 0, sizeof(float) * R * k2p));
    MC_CUDA(cudaMemcpy2D(d1.p, sizeof(float) * k1p, X1, sizeof(float) * K1, sizeof(float) * K1, R, cudaMemcpyDefault));
    MC_CUDA(cudaMemcpy2D(d2.p, sizeof(float) * k2p, X2, sizeof(float) * K2, sizeof(float) * K2, R, cudaMemcpyDefault));
    const float *x2 = same ? d1.as<float>() : d2.as<float>();
    if (tensor_cores)
      gemm_tn_tc(0, R, K1, K2, d1.as<float>(), k1p, x2, k2p, dc.as<float>(), K2, dp.as<float>(), de.as<int>(),
                 nullptr);
    else
      gemm_tn_simt(0, R, K1, K2, d1.as<float>(), k1p, x2, k2p, dc.as<float>(), K2, dp.as<float>(), nullptr, same);
    int herr = 0;
    MC_CUDA(cudaMemcpy(&herr, de.p, sizeof(int), cudaMemcpyDeviceToHost));
    MC_CUDA(cudaMemcpy(C, dc.p, sizeof(float) * K1 * K2, cudaMemcpyDefault));
    MC_CUDA(cudaDeviceSynchronize());
    if (herr) fail(MC_ETIMEOUT, "a bounded wait in the tensor-core panel Gram expired");
    return MC_OK;
  });
}

mc_status mc_gather_rate(mc_handle h, int trans, int k, int reps, double *gbs) {
  if (!h || !gbs || k < 1 || k > 128 || reps < 1) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    const int kp = (int)round_up(k, 4);
    const int64_t rows_in = trans ? h->m : h->n;
    const int *idx = trans ? h->ri.as<int>() : h->ci.as<int>();
    int dev = 0, sms = 0;
    MC_CUDA(cudaGetDevice(&dev));
    MC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 8;
    DBuf dp, ds;
    BufGuard g(h->alloc, {&dp, &ds});
    dp.reserve(h->alloc, sizeof(float) * rows_in * kp);
    ds.reserve(h->alloc, sizeof(float) * (size_t)grid * 256);
    MC_CUDA(cudaMemsetAsync(dp.p, 0, sizeof(float) * rows_in * kp, h->stream));
    cudaEvent_t e0, e1;
    MC_CUDA(cudaEventCreate(&e0));
    MC_CUDA(cudaEventCreate(&e1));
    gather_probe(h->stream, h->nnz, idx, dp.as<float>(), kp, kp, ds.as<float>(), grid);  // warm-up
    MC_CUDA(cudaEventRecord(e0, h->stream));
    for (int r = 0; r < reps; ++r) gather_probe(h->stream, h->nnz, idx, dp.as<float>(), kp, kp, ds.as<float>(), grid);
    MC_CUDA(cudaEventRecord(e1, h->stream));
    MC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gbs = ms > 0.f ? (double)h->nnz * kp * 4.0 * reps / (ms * 1e-3) / 1e9 : 0.0;
    return MC_OK;
  });
}

mc_status mc_spmm(mc_handle h, int trans, int k, const float *X, float *out) {
  if (!h || k < 1 || !X || !out) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    const int kp = (int)round_up(k, 4);
    const int64_t rin = trans ? h->m : h->n, rout = trans ? h->n : h->m;
    DBuf dx, dy;
    BufGuard g_bufs(h->alloc, {&dx, &dy});
    dx.reserve(h->alloc, sizeof(float) * rin * kp);
    dy.reserve(h->alloc, sizeof(float) * rout * kp);
    MC_CUDA(cudaMemsetAsync(dx.p, 0, sizeof(float) * rin * kp, h->stream));
    MC_CUDA(cudaMemcpy2DAsync(dx.p, sizeof(float) * kp, X, sizeof(float) * k, sizeof(float) * k, rin, cudaMemcpyDefault,
                              h->stream));
    if (trans) spmm_Yt(h, dx.as<float>(), kp, kp, dy.as<float>(), kp);
    else spmm_Y(h, dx.as<float>(), kp, kp, dy.as<float>(), kp);
    copy_out_2d(h->stream, out, k, dy.as<float>(), kp, rout);
    sync(h);
    dx.release(h->alloc);
    dy.release(h->alloc);
    sync(h);
    return MC_OK;
  });
}

mc_status mc_timing_enable(mc_handle h, int on) {
  if (!h || on < 0 || on > 2) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    sync(h);
    h->prof.reset();
    h->prof.on = on != 0;
    h->prof.mask = on == 2 ? (1u << MC_T_SPMM) | (1u << MC_T_SPMM_T) : ~0u;
    return MC_OK;
  });
}

mc_status mc_timing_read(mc_handle h, mc_timing *out) {
  if (!h || !out) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    if (h->side) MC_CUDA(cudaStreamSynchronize(h->side));  // events recorded there too
    sync(h);
    h->prof.resolve();
    for (int i = 0; i < MC_T_COUNT; ++i) out[i] = h->prof.acc[i];
    return MC_OK;
  });
}

mc_status mc_omega(int64_t n, int k, uint64_t seed, uint64_t call_id, int col0, float *out, uint32_t *words) {
  if (n < 0 || k < 1 || !out || col0 < 0) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    float *d = nullptr;
    uint32_t *w = nullptr;
    MC_CUDA(cudaMalloc(&d, sizeof(float) * std::max<int64_t>(n * k, 1)));
    if (words) MC_CUDA(cudaMalloc(&w, sizeof(uint32_t) * std::max<int64_t>(2 * n * k, 1)));
    launch_omega(0, n, k, k, seed, call_id, col0, d, w);
    MC_CUDA(cudaMemcpy(out, d, sizeof(float) * n * k, cudaMemcpyDefault));
    if (words) MC_CUDA(cudaMemcpy(words, w, sizeof(uint32_t) * 2 * n * k, cudaMemcpyDefault));
    cudaFree(d);
    if (w) cudaFree(w);
    return MC_OK;
  });
}

mc_status mc_eig_sym(int K, int kw, const float *A, float *lam, float *W) {
  if (K < 1 || K > kMaxKt || kw < 1 || kw > K || !A || !lam || !W) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    float *dA = nullptr, *dl = nullptr, *dW = nullptr;
    void *work = nullptr;
    MC_CUDA(cudaMalloc(&dA, sizeof(float) * K * K));
    MC_CUDA(cudaMalloc(&dl, sizeof(float) * kw));
    MC_CUDA(cudaMalloc(&dW, sizeof(float) * K * kw));
    MC_CUDA(cudaMalloc(&work, eig_work_bytes(K, kw)));
    MC_CUDA(cudaMemcpy(dA, A, sizeof(float) * K * K, cudaMemcpyDefault));
    eig_topk(0, K, kw, dA, K, dl, dW, kw, work);
    MC_CUDA(cudaMemcpy(lam, dl, sizeof(float) * kw, cudaMemcpyDefault));
    MC_CUDA(cudaMemcpy(W, dW, sizeof(float) * K * kw, cudaMemcpyDefault));
    cudaFree(dA);
    cudaFree(dl);
    cudaFree(dW);
    cudaFree(work);
    return MC_OK;
  });
}

mc_status mc_gram_tc(int64_t R, int K, const float *X, float *G) {
  if (R < 1 || K < 1 || K > 256 || !X || !G) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    const int kp = (int)round_up(K, 4);
    float *dX = nullptr, *dG = nullptr, *part = nullptr;
    int *derr = nullptr;
    MC_CUDA(cudaMalloc(&dX, sizeof(float) * R * kp));
    MC_CUDA(cudaMalloc(&dG, sizeof(float) * K * K));
    MC_CUDA(cudaMalloc(&part, sizeof(float) * gram_tc_scratch_floats(R, K)));
    MC_CUDA(cudaMalloc(&derr, sizeof(int)));
    MC_CUDA(cudaMemset(derr, 0, sizeof(int)));
    MC_CUDA(cudaMemset(dX, 0, sizeof(float) * R * kp));
    MC_CUDA(cudaMemcpy2D(dX, sizeof(float) * kp, X, sizeof(float) * K, sizeof(float) * K, R, cudaMemcpyDefault));
    gram_tc(0, R, K, dX, kp, dG, K, part, derr);
    int herr = 0;
    MC_CUDA(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
    MC_CUDA(cudaMemcpy(G, dG, sizeof(float) * K * K, cudaMemcpyDefault));
    cudaFree(dX);
    cudaFree(dG);
    cudaFree(part);
    cudaFree(derr);
    if (herr) fail(MC_ETIMEOUT, "a bounded wait in the tensor-core Gram expired");
    return MC_OK;
  });
}

mc_status mc_panel_gemm(int64_t R, int K, int N, const float *X, const float *W, float *Z, int tensor_cores) {
  if (R < 1 || K < 1 || N < 1 || !X || !W || !Z) return MC_EINVAL;
  const int kp = (int)round_up(K, 4);
  if (tensor_cores && !gemm_nn_tc_supported(R, K, N, reinterpret_cast<const void *>(256), kp)) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    DBuf dX, dW, dZ, de;
    Alloc a;
    BufGuard g(a, {&dX, &dW, &dZ, &de});
    dX.reserve(a, sizeof(float) * R * kp);
    dW.reserve(a, sizeof(float) * K * N);
    dZ.reserve(a, sizeof(float) * R * N);
    de.reserve(a, sizeof(int));
    MC_CUDA(cudaMemset(de.p, 0, sizeof(int)));
    MC_CUDA(cudaMemset(dX.p, 0, sizeof(float) * R * kp));
    MC_CUDA(cudaMemcpy2D(dX.p, sizeof(float) * kp, X, sizeof(float) * K, sizeof(float) * K, R, cudaMemcpyDefault));
    MC_CUDA(cudaMemcpy(dW.p, W, sizeof(float) * K * N, cudaMemcpyDefault));
    if (tensor_cores)
      gemm_nn_tc(0, R, K, N, dX.as<float>(), kp, dW.as<float>(), N, nullptr, 1.0f, 0.0f, dZ.as<float>(), N,
                 de.as<int>());
    else
      gemm_nn_simt(0, R, K, N, dX.as<float>(), kp, dW.as<float>(), N, nullptr, 1.0f, 0.0f, dZ.as<float>(), N);
    int herr = 0;
    MC_CUDA(cudaMemcpy(&herr, de.p, sizeof(int), cudaMemcpyDeviceToHost));
    MC_CUDA(cudaMemcpy(Z, dZ.p, sizeof(float) * R * N, cudaMemcpyDefault));
    MC_CUDA(cudaDeviceSynchronize());
    if (herr) fail(MC_ETIMEOUT, "a bounded wait in the tensor-core panel product expired");
    return MC_OK;
  });
}

mc_status mc_orth_block(int64_t R, int K, float *X, int ldx, const float *Qp, int ldq, int cols, float *out, int ldo,
                        void *stream) {
  if (R < 1 || K < 1 || K > kMaxKt || K % 4 != 0 || cols < 0 || cols % 4 != 0 || !X || !out || ldx < K ||
      ldo < K || ldx % 4 != 0 || ldo % 4 != 0 || (cols > 0 && (!Qp || ldq < cols || ldq % 4 != 0)))
    return MC_EINVAL;
  if (!is_device_ptr(X) || !is_device_ptr(out) || (cols > 0 && !is_device_ptr(Qp))) return MC_EINVAL;
  if (((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(Qp)) & 15u) != 0)
    return MC_EINVAL;
  return guarded([&]() -> mc_status {
    // a matrix-less handle carries the stream, the allocator and the scratch
    std::unique_ptr<mc_handle_s, void (*)(mc_handle)> h(new mc_handle_s, mc_destroy);
    h->stream = static_cast<cudaStream_t>(stream);
    h->alloc.stream = h->stream;
    h->m = R;
    h->flags.reserve(h->alloc, sizeof(int) * 8);
    MC_CUDA(cudaMemsetAsync(h->flags.p, 0, sizeof(int) * 8, h->stream));
    orth_step(h.get(), R, K, X, ldx, Qp, ldq, cols, out, ldo);
    sync(h.get());
    return MC_OK;
  });
}

mc_status mc_gram(int64_t R, int K, const float *X, float *G) {
  if (R < 1 || K < 1 || !X || !G) return MC_EINVAL;
  return guarded([&]() -> mc_status {
    const int kp = (int)round_up(K, 4);
    float *dX = nullptr, *dG = nullptr, *part = nullptr;
    MC_CUDA(cudaMalloc(&dX, sizeof(float) * R * kp));
    MC_CUDA(cudaMalloc(&dG, sizeof(float) * K * K));
    MC_CUDA(cudaMalloc(&part, sizeof(float) * gemm_tn_scratch_floats(R, K, K)));
    MC_CUDA(cudaMemset(dX, 0, sizeof(float) * R * kp));
    MC_CUDA(cudaMemcpy2D(dX, sizeof(float) * kp, X, sizeof(float) * K, sizeof(float) * K, R, cudaMemcpyDefault));
    gemm_tn(0, R, K, K, dX, kp, dX, kp, dG, K, true, part);
    MC_CUDA(cudaMemcpy(G, dG, sizeof(float) * K * K, cudaMemcpyDefault));
    cudaFree(dX);
    cudaFree(dG);
    cudaFree(part);
    return MC_OK;
  });
}

}  // extern "C"
