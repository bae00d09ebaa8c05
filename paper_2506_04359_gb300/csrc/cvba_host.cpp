// Host side of the C ABI declared in include/cvba.h: argument validation, the device
// layout of one bundle-adjustment window (observations sorted by landmark, keyframe,
// camera; (landmark, keyframe) pairs; work tiles), device memory and the CUDA graph that
// replays a whole LM solve.
#include <algorithm>
#include <climits>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cvba_internal.h"

using namespace cvba;

struct cvba_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  SideStream side;                              // overlapping work of an iteration
  cvba_precision prec = CVBA_FP64;
  std::string err;

  int C = 0, K = 0, M = 0, N = 0, P = 0, fixed_kf = 0;
  std::vector<double> intr, T_cb, poses, lms;
  std::vector<int32_t> wh;                      // image sizes (zeros when not given)
  bool have_rig = false, have_poses = false, have_lms = false, have_layout = false;

  std::vector<int32_t> lm_order, lm_rank, obs_order, lm_off;
  HostLayout hl;                                // host layout and its work arrays (reused)
  std::vector<int32_t> h_kf, h_cam, h_lm;       // caller's observations (for re-planning)
  std::vector<double> h_uv;
  int tune_lin_pairs = 0, tune_schur_lms = 0;   // 0: size-based defaults
  int chol_mode = 0;                            // 0 size-based, 1 cluster, 2 blocked
  std::vector<LinTile> lin_tiles;
  std::vector<SchurTile> schur_tiles, direct_tiles;
  std::vector<int32_t> act_blk;                 // RCS blocks the reduction writes
  struct Tables {                               // host tables of the layout, kept so that a window
    std::vector<int32_t> lm_blk, kf_tiles_off;  // of the same shape reuses their storage
    std::vector<int32_t> lin_kf_off, lin_kf_idx, lin_kf_slot, blk_tiles_off, blk_tiles;
    std::vector<int> win_lo, win_hi;
  } tb;

  struct Slot {
    void* p;
    size_t cap;
  };
  std::vector<Slot> arena;       // device buffers of the layout, reused when large enough
  size_t arena_next = 0;
  void* h_pin = nullptr;         // pinned host staging of the layout's uploads (kept, grown)
  size_t h_pin_bytes = 0;
  Dev d{};
  double* d_eval = nullptr;
  int32_t* d_lm_order = nullptr;
  cvba_iter* d_trace = nullptr;
  int trace_cap = 0;
  cudaGraphExec_t graph = nullptr;
  Dev graph_dev{};               // device view the graph was captured with
  struct Key {
    int iters = -1, reset = -1, refine = -1;
    double lam0 = 0, huber = 0, zmin = 0;
    bool operator==(const Key& o) const {
      return iters == o.iters && reset == o.reset && refine == o.refine && lam0 == o.lam0 && huber == o.huber &&
             zmin == o.zmin;
    }
  } graph_key;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cvba_status fail(cvba_ctx* c, cvba_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

cvba_status cuda_fail(cvba_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? CVBA_ERR_OOM : CVBA_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

bool all_finite(const double* p, size_t n) {
  const int T = host_threads();
  std::vector<char> ok((size_t)T, 1);              // per thread: no non-finite value seen
  parallel_for((int64_t)n, T, [&](int64_t i0, int64_t i1, int t) {
    for (int64_t i = i0; i < i1; ++i)
      if (!std::isfinite(p[i])) {
        ok[t] = 0;
        break;
      }
  });
  return std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; });
}

void drop_graph(cvba_ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->graph_key = cvba_ctx::Key{};
}

void free_device(cvba_ctx* c) {
  drop_graph(c);
  for (auto& s : c->arena) cudaFree(s.p);
  c->arena.clear();
  c->arena_next = 0;
  if (c->d_trace) cudaFree(c->d_trace);
  c->d_trace = nullptr;
  c->trace_cap = 0;
  c->d = Dev{};
  c->d_eval = nullptr;
  c->d_lm_order = nullptr;
  c->have_layout = false;
}

// Pinned host staging of at least `bytes` (kept by the context and grown when needed), so the
// layout's large uploads are asynchronous copies at the link's rate.
cudaError_t ensure_pinned(cvba_ctx* c, size_t bytes) {
  if (bytes <= c->h_pin_bytes) return cudaSuccess;
  if (c->h_pin) cudaFreeHost(c->h_pin);
  c->h_pin = nullptr;
  c->h_pin_bytes = 0;
  const cudaError_t e = cudaMallocHost(&c->h_pin, bytes);
  if (e == cudaSuccess) c->h_pin_bytes = bytes;
  return e;
}

// Next buffer of the layout: the slot used by the previous layout is kept when it is
// large enough, so re-loading a window of the same shape allocates nothing.
template <typename T>
cudaError_t dalloc(cvba_ctx* c, T** p, size_t n) {
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  const size_t idx = c->arena_next++;
  if (idx < c->arena.size() && c->arena[idx].cap >= bytes) {
    *p = static_cast<T*>(c->arena[idx].p);
    return cudaSuccess;
  }
  void* q = nullptr;
  if (idx < c->arena.size()) {
    cudaFree(c->arena[idx].p);
    c->arena[idx] = {nullptr, 0};
  }
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return e;
  if (idx < c->arena.size())
    c->arena[idx] = {q, bytes};
  else
    c->arena.push_back({q, bytes});
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

// Stream-ordered copies on the context's stream (which may be a caller's stream).
cudaError_t d2h(cvba_ctx* c, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}
cudaError_t h2d(cvba_ctx* c, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}

int read_cur(cvba_ctx* c) {
  int cur = 0;
  if (c->d.ctrl && d2h(c, &cur, &c->d.ctrl->cur, sizeof(int)) != cudaSuccess) cur = 0;
  return cur;
}

// FP32 copy of `n` doubles into a device mirror (mixed path only).
cudaError_t upload_f32(cvba_ctx* c, float* dst, const double* src, size_t n) {
  if (!dst) return cudaSuccess;
  std::vector<float> h(n);
  for (size_t i = 0; i < n; ++i) h[i] = (float)src[i];
  return h2d(c, dst, h.data(), n * sizeof(float));
}

cvba_status build_layout(cvba_ctx* c, const int32_t* kf, const int32_t* cam, const int32_t* lm, const double* uv) {
  const int K = c->K, C = c->C, M = c->M, N = c->N;
  HostLayout& HL = c->hl;
  // the previous layout's arrays are reused as this one's storage
  HL.lm_order.swap(c->lm_order);
  HL.lm_rank.swap(c->lm_rank);
  HL.obs_order.swap(c->obs_order);
  HL.lm_off.swap(c->lm_off);
  {
    std::string err;
    if (!compute_host_layout(K, C, M, N, c->fixed_kf, kf, cam, lm, HL, err))
      return fail(c, CVBA_ERR_INVALID_ARG, err);
  }
  c->lm_order.swap(HL.lm_order);
  c->lm_rank.swap(HL.lm_rank);
  c->obs_order.swap(HL.obs_order);
  c->lm_off.swap(HL.lm_off);
  std::vector<int32_t>& pair_kf = HL.pair_kf;
  std::vector<int32_t>& pair_lm = HL.pair_lm;
  std::vector<int32_t>& pair_obs = HL.pair_obs;
  std::vector<int32_t>& lm_pair = HL.lm_pair;
  std::vector<int32_t>& obs_cam = HL.obs_cam;
  const int P = (int)pair_kf.size();
  std::vector<int32_t>& lm_blk = c->tb.lm_blk;
  lm_blk.assign((size_t)M + 1, 0);
  {
    int64_t acc = 0;
    for (int j = 0; j < M; ++j) {
      const int64_t m = lm_pair[j + 1] - lm_pair[j];
      acc += m * (m - 1) / 2;
      if (acc > INT32_MAX) return fail(c, CVBA_ERR_INVALID_ARG, "too many pose-pair blocks");
      lm_blk[j + 1] = (int32_t)acc;
    }
  }
  std::vector<int32_t> kf_pb(K);
  for (int a = 0; a < K; ++a) kf_pb[a] = a == c->fixed_kf ? -1 : (a < c->fixed_kf ? a : a - 1);
  c->P = P;

  // --- tiles
  const int n_sm = 152;
  c->lin_tiles.clear();
  {
    const int target = c->tune_lin_pairs > 0 ? std::min(LIN_TILE_PAIRS, c->tune_lin_pairs)
                                             : std::max(32, std::min(LIN_TILE_PAIRS, (P + 2 * n_sm - 1) / (2 * n_sm)));
    int l0 = 0;
    while (l0 < M) {
      int l1 = l0;
      while (l1 < M) {
        const int np = lm_pair[l1 + 1] - lm_pair[l0];
        if (l1 > l0 && (np > target || l1 - l0 >= LIN_TILE_LMS)) break;
        ++l1;
      }
      LinTile t{l0, l1, lm_pair[l0], lm_pair[l1], 0, 0, 0, 0, 0, 0, 0, 0};
      t.o0 = pair_obs[t.p0];
      t.o1 = pair_obs[t.p1];
      c->lin_tiles.push_back(t);
      l0 = l1;
    }
    // each tile's keyframe range, from its pairs
    parallel_ranges((int64_t)c->lin_tiles.size(), [&](int64_t t0, int64_t t1, int) {
      for (int64_t ti = t0; ti < t1; ++ti) {
        LinTile& t = c->lin_tiles[ti];
        int lo = K, hi = -1;
        for (int q = t.p0; q < t.p1; ++q) {
          lo = std::min(lo, pair_kf[q]);
          hi = std::max(hi, pair_kf[q]);
        }
        t.kf_lo = hi >= 0 ? lo : 0;
        t.kf_n = hi >= 0 ? hi - lo + 1 : 0;
      }
    });
  }
  // the per-keyframe partials, keyframe-major: keyframe a owns the slots [kf_tiles_off[a],
  // kf_tiles_off[a + 1]) (12 values each), one per tile covering it, in tile order
  std::vector<int32_t>& kf_tiles_off = c->tb.kf_tiles_off;
  kf_tiles_off.assign((size_t)K + 1, 0);
  size_t kf_part_len = 0;
  {
    for (auto& t : c->lin_tiles) {
      t.part_off = -1;
      kf_part_len += (size_t)t.kf_n * 12;
      for (int a = t.kf_lo; a < t.kf_lo + t.kf_n; ++a) kf_tiles_off[a + 1]++;
    }
    for (int a = 0; a < K; ++a) kf_tiles_off[a + 1] += kf_tiles_off[a];
  }
  std::vector<int32_t>& lin_kf_off = c->tb.lin_kf_off;
  std::vector<int32_t>& lin_kf_idx = c->tb.lin_kf_idx;
  std::vector<int32_t>& lin_kf_slot = c->tb.lin_kf_slot;
  // per tile and keyframe of its range: the tile-local indices of that keyframe's pairs
  // (free keyframes only), in pair order, and the keyframe's partial slot for this tile.
  // Offsets by a sequential pass over the tiles (free-pair counts first, in parallel), the
  // lists filled in parallel, tile by tile.
  const int n_lt = (int)c->lin_tiles.size();
  {
    std::vector<int32_t> n_free((size_t)n_lt, 0);
    parallel_ranges(n_lt, [&](int64_t t0, int64_t t1, int) {
      for (int64_t ti = t0; ti < t1; ++ti) {
        const LinTile& t = c->lin_tiles[ti];
        int m = 0;
        for (int q = t.p0; q < t.p1; ++q) m += kf_pb[pair_kf[q]] >= 0 ? 1 : 0;
        n_free[ti] = m;
      }
    });
    int kfl = 0, kfi = 0;
    for (int ti = 0; ti < n_lt; ++ti) {
      LinTile& t = c->lin_tiles[ti];
      t.kfl_off = kfl;
      t.kfi0 = kfi;
      t.kfi_n = n_free[ti];
      kfl += t.kf_n + 1;
      kfi += n_free[ti];
    }
    lin_kf_off.assign((size_t)kfl, 0);
    lin_kf_slot.assign((size_t)kfl, 0);
    lin_kf_idx.resize((size_t)kfi);                // every entry is written below
  }
  {
    std::vector<int32_t> slot_fill(kf_tiles_off.begin(), kf_tiles_off.end() - 1);
    for (const LinTile& t : c->lin_tiles)            // slots in tile order per keyframe
      for (int a = t.kf_lo; a < t.kf_lo + t.kf_n; ++a) lin_kf_slot[t.kfl_off + (a - t.kf_lo)] = slot_fill[a]++;
  }
  parallel_ranges(n_lt, [&](int64_t t0, int64_t t1, int) {
    std::vector<int32_t> cnt;
    for (int64_t ti = t0; ti < t1; ++ti) {
      const LinTile& t = c->lin_tiles[ti];
      cnt.assign((size_t)t.kf_n + 1, 0);
      for (int q = t.p0; q < t.p1; ++q)
        if (kf_pb[pair_kf[q]] >= 0) cnt[pair_kf[q] - t.kf_lo + 1]++;
      for (int k = 0; k < t.kf_n; ++k) cnt[k + 1] += cnt[k];
      for (int k = 0; k <= t.kf_n; ++k) lin_kf_off[t.kfl_off + k] = t.kfi0 + cnt[k];
      for (int q = t.p0; q < t.p1; ++q)
        if (kf_pb[pair_kf[q]] >= 0) lin_kf_idx[t.kfi0 + cnt[pair_kf[q] - t.kf_lo]++] = q - t.p0;
    }
  });
  // Schur tiles: runs of landmarks (in internal order) with the same window [lo, hi] of
  // free keyframes, at most `target` landmarks; landmarks spanning more than SPAN_MAX free
  // keyframes go to direct tiles (<= SCHUR_TILE_PAIRS pairs, <= SCHUR_TILE_LMS landmarks).
  c->schur_tiles.clear();
  c->direct_tiles.clear();
  int max_span = 1;
  {
    // default: at most 96 landmarks per tile (at 100 keyframes x 32 cameras, 96 against 128:
    // group Schur 367 against 381 us, reduction 25 against 22 us)
    const int target = c->tune_schur_lms > 0 ? std::min(SCHUR_TILE_LMS, c->tune_schur_lms)
                                             : std::max(8, std::min(96, (M + n_sm - 1) / n_sm));
    std::vector<int>& lo = c->tb.win_lo;
    std::vector<int>& hi = c->tb.win_hi;
    lo.assign((size_t)M, INT32_MAX);
    hi.assign((size_t)M, -1);
    parallel_for(M, host_threads(), [&](int64_t j0, int64_t j1, int) {
      for (int64_t j = j0; j < j1; ++j)
        for (int q = lm_pair[j]; q < lm_pair[j + 1]; ++q) {
          const int pb = kf_pb[pair_kf[q]];
          if (pb < 0) continue;
          lo[j] = std::min(lo[j], pb);
          hi[j] = std::max(hi[j], pb);
        }
    });
    auto wide = [&](int j) { return hi[j] >= 0 && hi[j] - lo[j] + 1 > SPAN_MAX; };
    int l0 = 0;
    while (l0 < M) {
      int l1 = l0 + 1;
      SchurTile t{};
      if (wide(l0)) {
        while (l1 < M && wide(l1) && l1 - l0 < SCHUR_TILE_LMS &&
               lm_pair[l1 + 1] - lm_pair[l0] <= SCHUR_TILE_PAIRS)
          ++l1;
        t.direct = 1;
        t.k_lo = 0;
        t.span = K - 1;
      } else {
        while (l1 < M && l1 - l0 < target && !wide(l1) && lo[l1] == lo[l0] && hi[l1] == hi[l0]) ++l1;
        t.direct = 0;
        t.k_lo = hi[l0] >= 0 ? lo[l0] : 0;
        t.span = hi[l0] >= 0 ? hi[l0] - lo[l0] + 1 : 0;
        max_span = std::max(max_span, t.span);
      }
      t.l0 = l0;
      t.l1 = l1;
      t.p0 = lm_pair[l0];
      t.p1 = lm_pair[l1];
      t.b0 = lm_blk[l0];
      t.b1 = lm_blk[l1];
      t.part_off = -1;
      (t.direct ? c->direct_tiles : c->schur_tiles).push_back(t);
      l0 = l1;
    }
  }
  // window partial offsets and, per block (a >= b) of free keyframes, the covering tiles
  const int nfb = K - 1;
  const int n_blk = nfb * (nfb + 1) / 2;
  std::vector<int32_t>& blk_tiles_off = c->tb.blk_tiles_off;
  std::vector<int32_t>& blk_tiles = c->tb.blk_tiles;
  blk_tiles_off.assign((size_t)n_blk + 1, 0);
  size_t schur_part_len = 0;
  {
    for (auto& t : c->schur_tiles) {
      const size_t part = (size_t)t.span * (t.span + 1) * 18;   // [half block][18]
      if (schur_part_len + part > (size_t)INT32_MAX)
        return fail(c, CVBA_ERR_INVALID_ARG, "Schur partials exceed 2^31 entries");
      t.part_off = (int)schur_part_len;
      schur_part_len += part;
      for (int a = t.k_lo; a < t.k_lo + t.span; ++a)
        for (int b = t.k_lo; b <= a; ++b) blk_tiles_off[a * (a + 1) / 2 + b + 1]++;
    }
    for (int i = 0; i < n_blk; ++i) blk_tiles_off[i + 1] += blk_tiles_off[i];
    blk_tiles.resize(blk_tiles_off[n_blk]);         // every entry is written below
    std::vector<int32_t> fill(blk_tiles_off.begin(), blk_tiles_off.end() - 1);
    for (int ti = 0; ti < (int)c->schur_tiles.size(); ++ti) {
      const auto& t = c->schur_tiles[ti];
      for (int a = t.k_lo; a < t.k_lo + t.span; ++a)
        for (int b = t.k_lo; b <= a; ++b) {
          const int aa = a - t.k_lo, bb = b - t.k_lo;   // [half block][18] window layout
          blk_tiles[fill[a * (a + 1) / 2 + b]++] = t.part_off + 2 * (aa * (aa + 1) / 2 + bb) * 18;
        }
    }
  }
  // blocks of the reduced camera system that any tile touches (and every diagonal block):
  // the only ones the reduction writes; the others stay zero from the layout on
  {
    std::vector<char> act(n_blk, 0);
    for (int i = 0; i < n_blk; ++i) act[i] = blk_tiles_off[i + 1] > blk_tiles_off[i];
    for (int a = 0; a < nfb; ++a) act[a * (a + 1) / 2 + a] = 1;
    std::vector<int> fb;
    for (const auto& t : c->direct_tiles)
      for (int j = t.l0; j < t.l1; ++j) {
        fb.clear();
        for (int q = lm_pair[j]; q < lm_pair[j + 1]; ++q)
          if (kf_pb[pair_kf[q]] >= 0) fb.push_back(kf_pb[pair_kf[q]]);
        for (int x : fb)
          for (int y : fb)
            if (x >= y) act[x * (x + 1) / 2 + y] = 1;
      }
    c->act_blk.clear();
    for (int i = 0; i < n_blk; ++i)
      if (act[i]) c->act_blk.push_back(i);
  }

  // --- device buffers
  c->have_layout = false;
  c->arena_next = 0;
  const int n_c = 6 * (K - 1);
  const bool mixed = c->prec == CVBA_MIXED;
  Dev& d = c->d;
  d = Dev{};
  d.K = K;
  d.C = C;
  d.M = M;
  d.N = N;
  d.P = P;
  d.n_c = n_c;
  d.fixed_kf = c->fixed_kf;
  d.mixed = mixed ? 1 : 0;
  d.n_lin_tiles = (int)c->lin_tiles.size();
  d.n_schur_tiles = (int)c->schur_tiles.size();
  d.n_direct_tiles = (int)c->direct_tiles.size();
  d.max_span = max_span;
  double *rig, *pose0, *pose1, *lm0, *lm1;
  int32_t *ocam, *pkf, *plm, *pobs, *lpair, *lblk, *kpb;
  LinTile* lt;
  SchurTile* st;
  CK(dalloc(c, &rig, (size_t)C * RIG_STRIDE), "alloc rig");
  CK(dalloc(c, &pose0, (size_t)K * POSE_STRIDE), "alloc poses");
  CK(dalloc(c, &pose1, (size_t)K * POSE_STRIDE), "alloc poses");
  CK(dalloc(c, &lm0, (size_t)M * 3), "alloc landmarks");
  CK(dalloc(c, &lm1, (size_t)M * 3), "alloc landmarks");
  CK(dalloc(c, &ocam, N), "alloc obs");
  CK(dalloc(c, &pkf, P), "alloc pairs");
  CK(dalloc(c, &plm, P), "alloc pairs");
  CK(dalloc(c, &pobs, (size_t)P + 1), "alloc pairs");
  CK(dalloc(c, &lpair, (size_t)M + 1), "alloc lm offsets");
  CK(dalloc(c, &lblk, (size_t)M + 1), "alloc lm offsets");
  CK(dalloc(c, &kpb, K), "alloc kf map");
  CK(dalloc(c, &lt, c->lin_tiles.size()), "alloc tiles");
  CK(dalloc(c, &st, c->schur_tiles.size()), "alloc tiles");
  SchurTile* dtl;
  CK(dalloc(c, &dtl, c->direct_tiles.size()), "alloc tiles");
  d.direct_tiles = dtl;
  d.rig = rig;
  d.pose[0] = pose0;
  d.pose[1] = pose1;
  d.lm[0] = lm0;
  d.lm[1] = lm1;
  if (mixed) {
    float *rf, *pf0, *pf1, *lf0, *lf1, *dcf;
    CK(dalloc(c, &rf, (size_t)C * RIG_STRIDE), "alloc mirrors");
    CK(dalloc(c, &pf0, (size_t)K * POSE_STRIDE), "alloc mirrors");
    CK(dalloc(c, &pf1, (size_t)K * POSE_STRIDE), "alloc mirrors");
    CK(dalloc(c, &lf0, (size_t)M * 3), "alloc mirrors");
    CK(dalloc(c, &lf1, (size_t)M * 3), "alloc mirrors");
    CK(dalloc(c, &dcf, (size_t)n_c), "alloc mirrors");
    d.rig_f = rf;
    d.pose_f[0] = pf0;
    d.pose_f[1] = pf1;
    d.lm_f[0] = lf0;
    d.lm_f[1] = lf1;
    d.dc_f = dcf;
  }
  d.obs_cam = ocam;
  d.pair_kf = pkf;
  d.pair_lm = plm;
  d.pair_obs = pobs;
  d.lm_pair = lpair;
  d.lm_blk = lblk;
  d.kf_pb = kpb;
  d.lin_tiles = lt;
  d.schur_tiles = st;
  // the observation pixels (in slot order, FP32 on the mixed path) and the large index arrays
  // go through the context's pinned staging by asynchronous copies on the library's stream,
  // waited for once at the end of the layout
  const size_t uv_bytes = (size_t)N * 2 * (mixed ? sizeof(float) : sizeof(double));
  const size_t idx_bytes = ((size_t)N + 3 * (size_t)P + 1 + 2 * ((size_t)M + 1)) * sizeof(int32_t);
  const size_t state_bytes = ((size_t)C * RIG_STRIDE + (size_t)K * POSE_STRIDE + (size_t)M * 3) * (mixed ? 12 : 8);
  const size_t table_bytes = (size_t)M * 4 + (size_t)K * 4 + sizeof(Ctrl) + c->lin_tiles.size() * sizeof(LinTile) +
                             (c->schur_tiles.size() + c->direct_tiles.size()) * sizeof(SchurTile);
  const size_t list_bytes = (kf_tiles_off.size() + lin_kf_slot.size() + blk_tiles_off.size() + blk_tiles.size() +
                             lin_kf_off.size() + lin_kf_idx.size() + c->act_blk.size()) * sizeof(int32_t);
  CK(cudaStreamSynchronize(c->stream), "sync");     // no copy of an earlier layout still reads the staging
  // (fewer than 40 buffers are taken from the staging, each rounded up to 256 bytes)
  CK(ensure_pinned(c, uv_bytes + idx_bytes + state_bytes + table_bytes + list_bytes + 40 * 256), "pinned staging");
  char* const pin = static_cast<char*>(c->h_pin);
  size_t pin_off = 0;
  auto pin_take = [&](size_t bytes) {
    char* h = pin + pin_off;
    pin_off += (bytes + 255) / 256 * 256;
    return h;
  };
  auto stage = [&](void* dst, const void* src, size_t bytes) {
    char* h = pin_take(bytes);
    parallel_for((int64_t)bytes, host_threads(), [&](int64_t b0, int64_t b1, int) {
      std::memcpy(h + b0, static_cast<const char*>(src) + b0, (size_t)(b1 - b0));
    });
    return cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, c->stream);
  };
  if (mixed) {
    float* uvf;
    CK(dalloc(c, &uvf, (size_t)N * 2), "alloc obs");
    float* h = reinterpret_cast<float*>(pin_take(uv_bytes));
    parallel_for(N, host_threads(), [&](int64_t s0, int64_t s1, int) {
      for (int64_t s = s0; s < s1; ++s) {
        if (s + 16 < s1) __builtin_prefetch(uv + 2 * (size_t)c->obs_order[s + 16]);   // a random gather
        h[2 * s] = (float)uv[2 * (size_t)c->obs_order[s]];
        h[2 * s + 1] = (float)uv[2 * (size_t)c->obs_order[s] + 1];
      }
    });
    CK(cudaMemcpyAsync(uvf, h, uv_bytes, cudaMemcpyHostToDevice, c->stream), "upload obs");
    d.obs_uv = uvf;
    float* pl;
    CK(dalloc(c, &pl, (size_t)P * PAIR_LIN), "alloc pair lin");
    d.pair_lin = pl;
  } else {
    double* uvd;
    CK(dalloc(c, &uvd, (size_t)N * 2), "alloc obs");
    double* h = reinterpret_cast<double*>(pin_take(uv_bytes));
    parallel_for(N, host_threads(), [&](int64_t s0, int64_t s1, int) {
      for (int64_t s = s0; s < s1; ++s) {
        if (s + 16 < s1) __builtin_prefetch(uv + 2 * (size_t)c->obs_order[s + 16]);   // a random gather
        h[2 * s] = uv[2 * (size_t)c->obs_order[s]];
        h[2 * s + 1] = uv[2 * (size_t)c->obs_order[s] + 1];
      }
    });
    CK(cudaMemcpyAsync(uvd, h, uv_bytes, cudaMemcpyHostToDevice, c->stream), "upload obs");
    d.obs_uv = uvd;
    double* pl;
    CK(dalloc(c, &pl, (size_t)P * PAIR_LIN), "alloc pair lin");
    d.pair_lin = pl;
  }
  CK(dalloc(c, &d.lm_H, (size_t)M * 6), "alloc");
  CK(dalloc(c, &d.lm_g, (size_t)M * 3), "alloc");
  CK(dalloc(c, &d.kf_gp, (size_t)K * 6), "alloc");
  CK(dalloc(c, &d.kf_dp, (size_t)K * 6), "alloc");
  CK(dalloc(c, &d.lm_Vinv, (size_t)M * VINV_STRIDE), "alloc");
  CK(dalloc(c, &d.S, (size_t)n_c * n_c), "alloc RCS");
  CK(dalloc(c, &d.bS, (size_t)n_c), "alloc");
  CK(dalloc(c, &d.dc, (size_t)n_c), "alloc");
  // blocked factorisation of large systems: the factor and y in global memory (one element
  // each otherwise, so that the buffers keep their places in the arena)
  d.npw = (n_c + 31) / 32 * 32;
  d.chol_blocked = c->chol_mode == 2 || (c->chol_mode == 0 && n_c >= kCholBlockedMinN) ? 1 : 0;
  {
    // factor envelope: first free keyframe coupled with each free keyframe (through a shared
    // landmark), then per panel the last row whose first coupled column falls in or before it
    std::vector<int> first_blk(K, INT32_MAX);
    {
      const int T = host_threads();
      std::vector<int> part((size_t)T * K, INT32_MAX);   // per thread, merged by min
      parallel_for(M, T, [&](int64_t j0, int64_t j1, int t) {
        int* fb = part.data() + (size_t)t * K;
        for (int64_t j = j0; j < j1; ++j) {
          int lo = INT32_MAX;
          for (int q = lm_pair[j]; q < lm_pair[j + 1]; ++q)
            if (kf_pb[pair_kf[q]] >= 0) lo = std::min(lo, kf_pb[pair_kf[q]]);
          for (int q = lm_pair[j]; q < lm_pair[j + 1]; ++q) {
            const int pb = kf_pb[pair_kf[q]];
            if (pb >= 0) fb[pb] = std::min(fb[pb], lo);
          }
        }
      });
      for (int t = 0; t < T; ++t)
        for (int a = 0; a < K; ++a) first_blk[a] = std::min(first_blk[a], part[(size_t)t * K + a]);
    }
    const int npan = d.npw / 32;
    for (int pn = 0; pn < kMaxPanels; ++pn) d.panel_end[pn] = 0;
    for (int pn = 0; pn < npan; ++pn) {
      const int end_col = 32 * pn + 31;
      int last = 32 * (pn + 1) - 1;             // the panel itself
      for (int i = 32 * (pn + 1); i < n_c; ++i) {
        const int f = first_blk[i / 6] == INT32_MAX ? i : 6 * first_blk[i / 6];
        if (f <= end_col) last = i;
      }
      d.panel_end[pn] = (int16_t)std::min(d.npw, (last + 1 + 31) / 32 * 32);
    }
  }
  CK(dalloc(c, &d.Lw, d.chol_blocked ? (size_t)d.npw * d.npw : 1), "alloc");
  CK(dalloc(c, &d.Ldinv, d.chol_blocked ? (size_t)d.npw : 1), "alloc");
  CK(dalloc(c, &d.yw, d.chol_blocked ? (size_t)d.npw : 1), "alloc");
  CK(dalloc(c, &d.dp, (size_t)M * 3), "alloc");
  {
    double *kp, *sp;
    int32_t *kto, *kt, *bto, *bt;
    CK(dalloc(c, &kp, kf_part_len), "alloc");
    CK(dalloc(c, &sp, schur_part_len), "alloc");
    CK(dalloc(c, &kto, (size_t)K + 1), "alloc");
    CK(dalloc(c, &kt, lin_kf_slot.size()), "alloc");
    CK(dalloc(c, &bto, (size_t)n_blk + 1), "alloc");
    CK(dalloc(c, &bt, blk_tiles.size()), "alloc");
    CK(stage(kto, kf_tiles_off.data(), kf_tiles_off.size() * 4), "upload");
    if (!lin_kf_slot.empty()) CK(stage(kt, lin_kf_slot.data(), lin_kf_slot.size() * 4), "upload");
    CK(stage(bto, blk_tiles_off.data(), blk_tiles_off.size() * 4), "upload");
    if (!blk_tiles.empty()) CK(stage(bt, blk_tiles.data(), blk_tiles.size() * 4), "upload");
    int32_t *lko, *lki;
    CK(dalloc(c, &lko, lin_kf_off.size()), "alloc");
    CK(dalloc(c, &lki, std::max<size_t>(1, lin_kf_idx.size())), "alloc");
    if (!lin_kf_off.empty()) CK(stage(lko, lin_kf_off.data(), lin_kf_off.size() * 4), "upload");
    if (!lin_kf_idx.empty()) CK(stage(lki, lin_kf_idx.data(), lin_kf_idx.size() * 4), "upload");
    d.lin_kf_off = lko;
    d.lin_kf_idx = lki;
    d.kf_part = kp;
    d.schur_part = sp;
    d.kf_tiles_off = kto;
    d.lin_kf_slot = kt;
    d.blk_tiles_off = bto;
    d.blk_part_at = bt;
    d.n_blk = n_blk;
    int32_t* ab;
    CK(dalloc(c, &ab, c->act_blk.size()), "alloc");
    CK(stage(ab, c->act_blk.data(), c->act_blk.size() * 4), "upload");
    d.act_blk = ab;
    d.n_act = (int)c->act_blk.size();
  }
  CK(dalloc(c, &d.lin_part, (size_t)d.n_lin_tiles * 4), "alloc");
  CK(dalloc(c, &d.bs_part, (size_t)d.n_lin_tiles * 8), "alloc");
  CK(dalloc(c, &d.ctrl, 1), "alloc");
  CK(dalloc(c, &c->d_eval, 4), "alloc");
  CK(dalloc(c, &c->d_lm_order, M), "alloc");
  CK(stage(c->d_lm_order, c->lm_order.data(), (size_t)M * 4), "upload");
  d.trace = c->d_trace;
  // zero fills on the library's stream, ordered with the copies below and the solve
  CK(cudaMemsetAsync(d.S, 0, sizeof(double) * std::max<size_t>((size_t)n_c * n_c, 1), c->stream), "memset");
  CK(cudaMemsetAsync(d.dc, 0, sizeof(double) * std::max(n_c, 1), c->stream), "memset");
  CK(cudaMemsetAsync(d.dp, 0, sizeof(double) * (size_t)M * 3, c->stream), "memset");
  CK(cudaMemsetAsync(d.lin_part, 0, sizeof(double) * (size_t)d.n_lin_tiles * 4, c->stream), "memset");
  CK(cudaMemsetAsync(d.bs_part, 0, sizeof(double) * (size_t)d.n_lin_tiles * 8, c->stream), "memset");
  {
    Ctrl h{};
    h.cur = 0;
    h.lam = 1e-4;
    h.nu = 2.0;
    CK(stage(d.ctrl, &h, sizeof(Ctrl)), "upload ctrl");
  }
  // rig, poses and landmarks (internal order), and their FP32 mirrors, assembled in the staging
  double* righ = reinterpret_cast<double*>(pin_take((size_t)C * RIG_STRIDE * 8));
  for (int k = 0; k < C; ++k) {
    for (int i = 0; i < 4; ++i) righ[k * RIG_STRIDE + i] = c->intr[k * 4 + i];
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) righ[k * RIG_STRIDE + 4 + r * 3 + q] = c->T_cb[k * 12 + r * 4 + q];
      righ[k * RIG_STRIDE + 13 + r] = c->T_cb[k * 12 + r * 4 + 3];
    }
  }
  double* poseh = reinterpret_cast<double*>(pin_take((size_t)K * POSE_STRIDE * 8));
  for (int a = 0; a < K; ++a)
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) poseh[a * POSE_STRIDE + r * 3 + q] = c->poses[a * 12 + r * 4 + q];
      poseh[a * POSE_STRIDE + 9 + r] = c->poses[a * 12 + r * 4 + 3];
    }
  double* lmh = reinterpret_cast<double*>(pin_take((size_t)M * 3 * 8));
  parallel_for(M, host_threads(), [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i)
      for (int k = 0; k < 3; ++k) lmh[i * 3 + k] = c->lms[(size_t)c->lm_order[i] * 3 + k];
  });
  CK(cudaMemcpyAsync(rig, righ, (size_t)C * RIG_STRIDE * 8, cudaMemcpyHostToDevice, c->stream), "upload rig");
  CK(cudaMemcpyAsync(pose0, poseh, (size_t)K * POSE_STRIDE * 8, cudaMemcpyHostToDevice, c->stream), "upload poses");
  CK(cudaMemcpyAsync(lm0, lmh, (size_t)M * 3 * 8, cudaMemcpyHostToDevice, c->stream), "upload landmarks");
  if (mixed) {
    auto mirror = [&](float* dst, const double* src, size_t n) {
      float* h = reinterpret_cast<float*>(pin_take(n * 4));
      parallel_for((int64_t)n, host_threads(), [&](int64_t e0, int64_t e1, int) {
        for (int64_t e = e0; e < e1; ++e) h[e] = (float)src[e];
      });
      return cudaMemcpyAsync(dst, h, n * 4, cudaMemcpyHostToDevice, c->stream);
    };
    CK(mirror(const_cast<float*>(d.rig_f), righ, (size_t)C * RIG_STRIDE), "upload mirrors");
    CK(mirror(d.pose_f[0], poseh, (size_t)K * POSE_STRIDE), "upload mirrors");
    CK(mirror(d.lm_f[0], lmh, (size_t)M * 3), "upload mirrors");
  }
  CK(stage(ocam, obs_cam.data(), (size_t)N * 4), "upload");
  CK(stage(pkf, pair_kf.data(), (size_t)P * 4), "upload");
  CK(stage(plm, pair_lm.data(), (size_t)P * 4), "upload");
  CK(stage(pobs, pair_obs.data(), ((size_t)P + 1) * 4), "upload");
  CK(stage(lpair, lm_pair.data(), ((size_t)M + 1) * 4), "upload");
  CK(stage(lblk, lm_blk.data(), ((size_t)M + 1) * 4), "upload");
  CK(stage(kpb, kf_pb.data(), (size_t)K * 4), "upload");
  CK(stage(lt, c->lin_tiles.data(), c->lin_tiles.size() * sizeof(LinTile)), "upload");
  if (!c->schur_tiles.empty()) CK(stage(st, c->schur_tiles.data(), c->schur_tiles.size() * sizeof(SchurTile)), "upload");
  if (!c->direct_tiles.empty())
    CK(stage(dtl, c->direct_tiles.data(), c->direct_tiles.size() * sizeof(SchurTile)), "upload");
  CK(cudaStreamSynchronize(c->stream), "upload");   // the staging is free again
  c->have_layout = true;
  return CVBA_OK;
}

// Poses and / or landmarks replaced after the layout exists: written into the current state
// buffer (FP64, and the FP32 mirrors on the mixed path) from the context's pinned staging, by
// asynchronous copies waited for once.  Only what was replaced is written.
cvba_status upload_state(cvba_ctx* c, bool poses, bool lms) {
  const int cur = read_cur(c);                     // (waits for the stream: the staging is free)
  const int K = c->K, M = c->M;
  const size_t need = (poses ? (size_t)K * POSE_STRIDE * 12 : 0) + (lms ? (size_t)M * 3 * 12 : 0) + 4 * 256;
  CK(ensure_pinned(c, need), "pinned staging");
  char* const pin = static_cast<char*>(c->h_pin);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* h = pin + off;
    off += (bytes + 255) / 256 * 256;
    return h;
  };
  if (poses) {
    double* ph = reinterpret_cast<double*>(take((size_t)K * POSE_STRIDE * 8));
    for (int a = 0; a < K; ++a)
      for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) ph[a * POSE_STRIDE + r * 3 + q] = c->poses[a * 12 + r * 4 + q];
        ph[a * POSE_STRIDE + 9 + r] = c->poses[a * 12 + r * 4 + 3];
      }
    CK(cudaMemcpyAsync(c->d.pose[cur], ph, (size_t)K * POSE_STRIDE * 8, cudaMemcpyHostToDevice, c->stream), "upload");
    if (c->d.pose_f[cur]) {
      float* pf = reinterpret_cast<float*>(take((size_t)K * POSE_STRIDE * 4));
      for (int e = 0; e < K * POSE_STRIDE; ++e) pf[e] = (float)ph[e];
      CK(cudaMemcpyAsync(c->d.pose_f[cur], pf, (size_t)K * POSE_STRIDE * 4, cudaMemcpyHostToDevice, c->stream),
         "upload mirrors");
    }
  }
  if (lms) {
    double* lh = reinterpret_cast<double*>(take((size_t)M * 3 * 8));
    float* lf = c->d.lm_f[cur] ? reinterpret_cast<float*>(take((size_t)M * 3 * 4)) : nullptr;
    parallel_for(M, host_threads(), [&](int64_t i0, int64_t i1, int) {
      for (int64_t i = i0; i < i1; ++i)
        for (int k = 0; k < 3; ++k) {
          const double v = c->lms[(size_t)c->lm_order[i] * 3 + k];
          lh[i * 3 + k] = v;
          if (lf) lf[i * 3 + k] = (float)v;
        }
    });
    CK(cudaMemcpyAsync(c->d.lm[cur], lh, (size_t)M * 3 * 8, cudaMemcpyHostToDevice, c->stream), "upload");
    if (lf) CK(cudaMemcpyAsync(c->d.lm_f[cur], lf, (size_t)M * 3 * 4, cudaMemcpyHostToDevice, c->stream), "upload mirrors");
  }
  CK(cudaStreamSynchronize(c->stream), "sync");
  return CVBA_OK;
}

}  // namespace

extern "C" {

const char* cvba_status_string(cvba_status s) {
  switch (s) {
    case CVBA_OK: return "ok";
    case CVBA_ERR_INVALID_ARG: return "invalid argument";
    case CVBA_ERR_INDEX: return "index out of range";
    case CVBA_ERR_NONFINITE: return "non-finite input";
    case CVBA_ERR_CUDA: return "CUDA error";
    case CVBA_ERR_OOM: return "out of device memory";
    case CVBA_ERR_NOT_PD: return "not positive definite";
    case CVBA_ERR_TIMEOUT: return "device wait timed out";
    case CVBA_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* cvba_last_error(const cvba_ctx* c) { return c ? c->err.c_str() : ""; }

cvba_status cvba_create(cvba_ctx** out, int device, void* stream, cvba_precision prec) {
  if (!out) return CVBA_ERR_INVALID_ARG;
  *out = nullptr;
  if (prec != CVBA_FP64 && prec != CVBA_MIXED) return CVBA_ERR_INVALID_ARG;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return CVBA_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return CVBA_ERR_CUDA;   // built for sm_103a only
  cvba_ctx* c = new cvba_ctx();
  c->device = device;
  c->prec = prec;
  DeviceGuard g(device);
  cudaError_t e = set_kernel_attributes();
  if (e == cudaSuccess) {
    if (stream) {
      c->stream = static_cast<cudaStream_t>(stream);
    } else {
      e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      c->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side.s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->side.join) cudaEventDestroy(c->side.join);
    if (c->side.fork) cudaEventDestroy(c->side.fork);
    if (c->side.s) cudaStreamDestroy(c->side.s);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return CVBA_ERR_CUDA;
  }
  *out = c;
  return CVBA_OK;
}

void cvba_destroy(cvba_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->side.s) cudaStreamSynchronize(c->side.s);
    free_device(c);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    c->h_pin = nullptr;
    c->h_pin_bytes = 0;
    if (c->side.join) cudaEventDestroy(c->side.join);
    if (c->side.fork) cudaEventDestroy(c->side.fork);
    if (c->side.s) cudaStreamDestroy(c->side.s);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  }
  delete c;
}

cvba_status cvba_set_rig(cvba_ctx* c, int n_cams, const double* intr, const double* T_cb, const int32_t* wh) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (n_cams < 1 || n_cams > C_MAX || !intr || !T_cb)
    return fail(c, CVBA_ERR_INVALID_ARG, "set_rig: need 1 <= n_cams <= 64 and non-NULL arrays");
  if (!all_finite(intr, (size_t)n_cams * 4) || !all_finite(T_cb, (size_t)n_cams * 12))
    return fail(c, CVBA_ERR_NONFINITE, "set_rig: non-finite value");
  if (wh)
    for (int k = 0; k < 2 * n_cams; ++k)
      if (wh[k] <= 0) return fail(c, CVBA_ERR_INVALID_ARG, "set_rig: image sizes must be positive");
  DeviceGuard g(c->device);
  if (c->have_layout && n_cams != c->C) c->have_layout = false;
  c->C = n_cams;
  c->intr.assign(intr, intr + (size_t)n_cams * 4);
  c->T_cb.assign(T_cb, T_cb + (size_t)n_cams * 12);
  if (wh)
    c->wh.assign(wh, wh + (size_t)n_cams * 2);
  else
    c->wh.assign((size_t)n_cams * 2, 0);
  c->have_rig = true;
  if (c->have_layout) {
    std::vector<double> righ((size_t)c->C * RIG_STRIDE);
    for (int k = 0; k < c->C; ++k) {
      for (int i = 0; i < 4; ++i) righ[k * RIG_STRIDE + i] = c->intr[k * 4 + i];
      for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) righ[k * RIG_STRIDE + 4 + r * 3 + q] = c->T_cb[k * 12 + r * 4 + q];
        righ[k * RIG_STRIDE + 13 + r] = c->T_cb[k * 12 + r * 4 + 3];
      }
    }
    CK(h2d(c, const_cast<double*>(c->d.rig), righ.data(), righ.size() * 8), "upload rig");
    CK(upload_f32(c, const_cast<float*>(c->d.rig_f), righ.data(), righ.size()), "upload rig");
  }
  return CVBA_OK;
}

cvba_status cvba_get_rig(cvba_ctx* c, double* intr, double* T_cb, int32_t* wh) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (!c->have_rig) return fail(c, CVBA_ERR_STATE, "get_rig: no rig");
  if (intr) std::copy(c->intr.begin(), c->intr.end(), intr);
  if (T_cb) std::copy(c->T_cb.begin(), c->T_cb.end(), T_cb);
  if (wh) std::copy(c->wh.begin(), c->wh.end(), wh);
  return CVBA_OK;
}

cvba_status cvba_set_poses(cvba_ctx* c, int n_kf, const double* T_bw, int fixed_kf) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (n_kf < 2 || n_kf > K_MAX || !T_bw)
    return fail(c, CVBA_ERR_INVALID_ARG, "set_poses: need 2 <= n_kf <= 256 and a non-NULL array");
  if (fixed_kf < 0 || fixed_kf >= n_kf) return fail(c, CVBA_ERR_INDEX, "set_poses: fixed_kf out of range");
  if (!all_finite(T_bw, (size_t)n_kf * 12)) return fail(c, CVBA_ERR_NONFINITE, "set_poses: non-finite value");
  DeviceGuard g(c->device);
  if (c->have_layout && (n_kf != c->K || fixed_kf != c->fixed_kf)) c->have_layout = false;
  c->K = n_kf;
  c->fixed_kf = fixed_kf;
  c->poses.assign(T_bw, T_bw + (size_t)n_kf * 12);
  c->have_poses = true;
  if (c->have_layout) return upload_state(c, true, false);
  return CVBA_OK;
}

cvba_status cvba_set_landmarks(cvba_ctx* c, int n_lm, const double* p_w) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (n_lm < 1 || !p_w) return fail(c, CVBA_ERR_INVALID_ARG, "set_landmarks: need n_lm >= 1 and a non-NULL array");
  if (!all_finite(p_w, (size_t)n_lm * 3)) return fail(c, CVBA_ERR_NONFINITE, "set_landmarks: non-finite value");
  DeviceGuard g(c->device);
  if (c->have_layout && n_lm != c->M) c->have_layout = false;
  c->M = n_lm;
  c->lms.resize((size_t)n_lm * 3);
  parallel_for((int64_t)n_lm * 3, host_threads(), [&](int64_t e0, int64_t e1, int) {
    std::copy(p_w + e0, p_w + e1, c->lms.begin() + e0);
  });
  c->have_lms = true;
  if (c->have_layout) return upload_state(c, false, true);
  return CVBA_OK;
}

cvba_status cvba_set_observations(cvba_ctx* c, int n_obs, const int32_t* kf, const int32_t* cam,
                                  const int32_t* lm, const double* uv) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (!c->have_rig || !c->have_poses || !c->have_lms)
    return fail(c, CVBA_ERR_STATE, "set_observations: set rig, poses and landmarks first");
  if (n_obs < 1 || !kf || !cam || !lm || !uv)
    return fail(c, CVBA_ERR_INVALID_ARG, "set_observations: need n_obs >= 1 and non-NULL arrays");
  {
    // index and finiteness checks, in parallel; the first failing observation is reported
    const int T = host_threads();
    std::vector<int64_t> bad_idx((size_t)T, INT64_MAX), bad_uv((size_t)T, INT64_MAX);
    parallel_for(n_obs, T, [&](int64_t n0, int64_t n1, int t) {
      for (int64_t n = n0; n < n1; ++n) {
        if (kf[n] < 0 || kf[n] >= c->K || cam[n] < 0 || cam[n] >= c->C || lm[n] < 0 || lm[n] >= c->M) {
          bad_idx[t] = std::min(bad_idx[t], n);
          break;
        }
      }
      for (int64_t n = n0; n < n1; ++n)
        if (!std::isfinite(uv[2 * n]) || !std::isfinite(uv[2 * n + 1])) {
          bad_uv[t] = std::min(bad_uv[t], n);
          break;
        }
    });
    const int64_t bi = *std::min_element(bad_idx.begin(), bad_idx.end());
    const int64_t bu = *std::min_element(bad_uv.begin(), bad_uv.end());
    if (bi != INT64_MAX)
      return fail(c, CVBA_ERR_INDEX, "set_observations: index out of range at observation " + std::to_string(bi));
    if (bu != INT64_MAX) return fail(c, CVBA_ERR_NONFINITE, "set_observations: non-finite uv");
  }
  DeviceGuard g(c->device);
  c->N = n_obs;
  c->h_kf.resize(n_obs);
  c->h_cam.resize(n_obs);
  c->h_lm.resize(n_obs);
  c->h_uv.resize(2 * (size_t)n_obs);
  parallel_for(n_obs, host_threads(), [&](int64_t n0, int64_t n1, int) {   // kept for re-planning
    std::copy(kf + n0, kf + n1, c->h_kf.begin() + n0);
    std::copy(cam + n0, cam + n1, c->h_cam.begin() + n0);
    std::copy(lm + n0, lm + n1, c->h_lm.begin() + n0);
    std::copy(uv + 2 * n0, uv + 2 * n1, c->h_uv.begin() + 2 * n0);
  });
  return build_layout(c, kf, cam, lm, uv);
}

namespace {
// Re-plan the layout with the same observations, keeping the state on the device.
cvba_status replan(cvba_ctx* c) {
  if (!c->have_layout) return CVBA_OK;
  DeviceGuard g(c->device);
  // re-plan with the same observations; the state on the device is kept
  const int cur = read_cur(c);
  std::vector<double> poses((size_t)c->K * 12), lms((size_t)c->M * 3);
  cvba_status st = cvba_get_poses(c, poses.data());
  if (st == CVBA_OK) st = cvba_get_landmarks(c, lms.data());
  if (st != CVBA_OK) return st;
  double lam = 1e-4, nu = 2.0;
  cvba_get_damping(c, &lam, &nu);
  c->poses = poses;
  c->lms = lms;
  (void)cur;
  st = build_layout(c, c->h_kf.data(), c->h_cam.data(), c->h_lm.data(), c->h_uv.data());
  if (st == CVBA_OK) st = cvba_set_damping(c, lam, nu);
  return st;
}
}  // namespace

cvba_status cvba_set_tuning(cvba_ctx* c, int lin_tile_pairs, int schur_tile_landmarks) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (lin_tile_pairs < 0 || schur_tile_landmarks < 0)
    return fail(c, CVBA_ERR_INVALID_ARG, "set_tuning: sizes must be >= 0 (0 = default)");
  c->tune_lin_pairs = lin_tile_pairs;
  c->tune_schur_lms = schur_tile_landmarks;
  return replan(c);
}

cvba_status cvba_set_chol_mode(cvba_ctx* c, int mode) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return fail(c, CVBA_ERR_INVALID_ARG, "set_chol_mode: mode must be 0, 1 or 2");
  c->chol_mode = mode;
  return replan(c);
}

namespace {
bool opts_ok(const cvba_opts* o) {
  return o->iters >= 0 && o->huber_delta > 0.0 && std::isfinite(o->huber_delta) && std::isfinite(o->z_min) &&
         (!o->reset_lambda || (o->lambda0 > 0.0 && std::isfinite(o->lambda0))) && o->refine <= 8;
}

cvba_ctx::Key make_key(const cvba_opts* o, bool mixed) {
  cvba_ctx::Key key;
  key.iters = o->iters;
  key.reset = o->reset_lambda ? 1 : 0;
  key.refine = o->refine < 0 ? (mixed ? 1 : 0) : o->refine;
  key.lam0 = o->lambda0;
  key.huber = o->huber_delta;
  key.zmin = o->z_min;
  return key;
}

cvba_status enqueue_solve(cvba_ctx* c, const cvba_opts* o) {
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "solve: set_observations first");
  if (!opts_ok(o)) return fail(c, CVBA_ERR_INVALID_ARG, "solve: bad options");
  if (o->iters == 0) return CVBA_OK;
  if (o->iters > c->trace_cap) {
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (c->d_trace) cudaFree(c->d_trace);
    c->d_trace = nullptr;
    c->trace_cap = 0;
    CK(cudaMalloc(&c->d_trace, sizeof(cvba_iter) * (size_t)o->iters), "alloc trace");
    c->trace_cap = o->iters;
  }
  c->d.trace = c->d_trace;
  const cvba_ctx::Key key = make_key(o, c->prec == CVBA_MIXED);
  if (!c->graph || !(key == c->graph_key) || std::memcmp(&c->graph_dev, &c->d, sizeof(Dev)) != 0) {
    drop_graph(c);
    cudaGraph_t gr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_solve_init(c->d, o->lambda0, o->huber_delta, o->z_min, o->iters, key.reset, key.refine,
                                       c->stream);
    for (int it = 0; it < o->iters && e == cudaSuccess; ++it) e = enqueue_iteration(c->d, c->stream, nullptr, &c->side);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
    if (e != cudaSuccess) return cuda_fail(c, e, "enqueue solve");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
    e = cudaGraphInstantiate(&c->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(c, e, "instantiate graph");
    c->graph_key = key;
    std::memcpy(&c->graph_dev, &c->d, sizeof(Dev));
  }
  CK(cudaGraphLaunch(c->graph, c->stream), "launch solve");
  return CVBA_OK;
}
}  // namespace

cvba_status cvba_solve(cvba_ctx* c, const cvba_opts* o, cvba_iter* trace) {
  if (!c || !o) return CVBA_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  cvba_status st = enqueue_solve(c, o);
  if (st != CVBA_OK || o->iters == 0) return st;
  if (trace)
    CK(cudaMemcpyAsync(trace, c->d_trace, sizeof(cvba_iter) * (size_t)o->iters, cudaMemcpyDeviceToHost, c->stream),
       "copy trace");
  CK(cudaStreamSynchronize(c->stream), "solve");
  return CVBA_OK;
}

cvba_status cvba_solve_async(cvba_ctx* c, const cvba_opts* o) {
  if (!c || !o) return CVBA_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  return enqueue_solve(c, o);
}

cvba_status cvba_get_trace(cvba_ctx* c, cvba_iter* trace, int n) {
  if (!c || !trace || n < 0) return CVBA_ERR_INVALID_ARG;
  if (n > c->trace_cap) return fail(c, CVBA_ERR_INVALID_ARG, "get_trace: more records than the last solve");
  if (n == 0) return CVBA_OK;
  DeviceGuard g(c->device);
  CK(d2h(c, trace, c->d_trace, sizeof(cvba_iter) * (size_t)n), "copy trace");
  return CVBA_OK;
}

cvba_status cvba_set_poses_dev(cvba_ctx* c, const double* T_bw) {
  if (!c || !T_bw) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "set_poses_dev: set_observations first");
  DeviceGuard g(c->device);
  CK(enqueue_state_io(c->d, 0, const_cast<double*>(T_bw), c->d_lm_order, c->stream), "set poses");
  return CVBA_OK;
}

cvba_status cvba_set_landmarks_dev(cvba_ctx* c, const double* p_w) {
  if (!c || !p_w) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "set_landmarks_dev: set_observations first");
  DeviceGuard g(c->device);
  CK(enqueue_state_io(c->d, 1, const_cast<double*>(p_w), c->d_lm_order, c->stream), "set landmarks");
  return CVBA_OK;
}

cvba_status cvba_get_poses_dev(cvba_ctx* c, double* T_bw) {
  if (!c || !T_bw) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "get_poses_dev: set_observations first");
  DeviceGuard g(c->device);
  CK(enqueue_state_io(c->d, 2, T_bw, c->d_lm_order, c->stream), "get poses");
  return CVBA_OK;
}

cvba_status cvba_get_landmarks_dev(cvba_ctx* c, double* p_w) {
  if (!c || !p_w) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "get_landmarks_dev: set_observations first");
  DeviceGuard g(c->device);
  CK(enqueue_state_io(c->d, 3, p_w, c->d_lm_order, c->stream), "get landmarks");
  return CVBA_OK;
}

cvba_status cvba_profile_iteration(cvba_ctx* c, const cvba_opts* o, int reps, float* ms, int* n_parts) {
  if (!c || !o || reps < 1) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "profile: set_observations first");
  const int np = profile_parts();
  if (n_parts) *n_parts = np;
  if (!ms) return CVBA_OK;
  DeviceGuard g(c->device);
  cvba_opts one = *o;
  one.iters = reps;
  if (reps > c->trace_cap) {
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (c->d_trace) cudaFree(c->d_trace);
    c->d_trace = nullptr;
    c->trace_cap = 0;
    CK(cudaMalloc(&c->d_trace, sizeof(cvba_iter) * (size_t)reps), "alloc trace");
    c->trace_cap = reps;
  }
  c->d.trace = c->d_trace;
  std::vector<cudaEvent_t> ev((size_t)np + 1);
  for (auto& e : ev) CK(cudaEventCreate(&e), "event");
  std::vector<double> acc(np, 0.0);
  if (!opts_ok(&one)) return fail(c, CVBA_ERR_INVALID_ARG, "profile: bad options");
  const int refine = make_key(&one, c->prec == CVBA_MIXED).refine;
  cvba_status st = CVBA_OK;
  for (int r = 0; r < reps && st == CVBA_OK; ++r) {
    // each repetition starts a one-iteration solve from the current state, so every one
    // relinearises (a rejected step would otherwise skip the next linearisation)
    cudaError_t e = enqueue_solve_init(c->d, one.lambda0, one.huber_delta, one.z_min, 1, one.reset_lambda, refine,
                                       c->stream);
    if (e == cudaSuccess) e = enqueue_iteration(c->d, c->stream, ev.data(), &c->side);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[np]);
    if (e != cudaSuccess) {
      st = cuda_fail(c, e, "profile iteration");
      break;
    }
    for (int k = 0; k < np; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != CVBA_OK) return st;
  for (int k = 0; k < np; ++k) ms[k] = (float)(acc[k] / reps);
  return CVBA_OK;
}

const char* cvba_profile_names(void) { return profile_names(); }

cvba_status cvba_evaluate(cvba_ctx* c, double huber, double zmin, double* cost, double* rms, int* nv, int* ni) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "evaluate: set_observations first");
  if (!(huber > 0.0) || !std::isfinite(zmin)) return fail(c, CVBA_ERR_INVALID_ARG, "evaluate: bad options");
  DeviceGuard g(c->device);
  CK(enqueue_evaluate(c->d, huber, zmin, c->d_eval, c->stream), "evaluate");
  double h[4];
  CK(cudaMemcpyAsync(h, c->d_eval, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy");
  CK(cudaStreamSynchronize(c->stream), "evaluate");
  if (cost) *cost = h[0];
  if (rms) *rms = h[2] > 0 ? std::sqrt(h[1] / h[2]) : 0.0;
  if (nv) *nv = (int)h[2];
  if (ni) *ni = (int)h[3];
  return CVBA_OK;
}

cvba_status cvba_get_poses(cvba_ctx* c, double* T_bw) {
  if (!c || !T_bw) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) {
    if (!c->have_poses) return fail(c, CVBA_ERR_STATE, "get_poses: no poses");
    std::copy(c->poses.begin(), c->poses.end(), T_bw);
    return CVBA_OK;
  }
  DeviceGuard g(c->device);
  const int cur = read_cur(c);
  std::vector<double> h((size_t)c->K * POSE_STRIDE);
  CK(d2h(c, h.data(), c->d.pose[cur], h.size() * 8), "copy poses");
  for (int a = 0; a < c->K; ++a)
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) T_bw[a * 12 + r * 4 + q] = h[a * POSE_STRIDE + r * 3 + q];
      T_bw[a * 12 + r * 4 + 3] = h[a * POSE_STRIDE + 9 + r];
    }
  return CVBA_OK;
}

cvba_status cvba_get_landmarks(cvba_ctx* c, double* p_w) {
  if (!c || !p_w) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) {
    if (!c->have_lms) return fail(c, CVBA_ERR_STATE, "get_landmarks: no landmarks");
    std::copy(c->lms.begin(), c->lms.end(), p_w);
    return CVBA_OK;
  }
  DeviceGuard g(c->device);
  const int cur = read_cur(c);                     // (waits for the stream: the staging is free)
  const size_t bytes = (size_t)c->M * 3 * 8;
  CK(ensure_pinned(c, bytes), "pinned staging");
  CK(d2h(c, c->h_pin, c->d.lm[cur], bytes), "copy landmarks");
  const double* h = static_cast<const double*>(c->h_pin);
  parallel_for(c->M, host_threads(), [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i)
      for (int k = 0; k < 3; ++k) p_w[(size_t)c->lm_order[i] * 3 + k] = h[(size_t)i * 3 + k];
  });
  return CVBA_OK;
}

cvba_status cvba_get_increment(cvba_ctx* c, double* dx) {
  if (!c || !dx) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "get_increment: no layout");
  DeviceGuard g(c->device);
  const int n_c = c->d.n_c;
  CK(d2h(c, dx, c->d.dc, sizeof(double) * n_c), "copy dc");
  std::vector<double> h((size_t)c->M * 3);
  CK(d2h(c, h.data(), c->d.dp, h.size() * 8), "copy dp");
  for (int i = 0; i < c->M; ++i)
    for (int k = 0; k < 3; ++k) dx[n_c + (size_t)c->lm_order[i] * 3 + k] = h[(size_t)i * 3 + k];
  return CVBA_OK;
}

cvba_status cvba_get_damping(cvba_ctx* c, double* lam, double* nu) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "get_damping: no layout");
  DeviceGuard g(c->device);
  Ctrl h;
  CK(d2h(c, &h, c->d.ctrl, sizeof(Ctrl)), "copy ctrl");
  if (lam) *lam = h.lam;
  if (nu) *nu = h.nu;
  return CVBA_OK;
}

cvba_status cvba_set_damping(cvba_ctx* c, double lam, double nu) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "set_damping: no layout");
  if (!(lam > 0.0) || !(nu >= 1.0) || !std::isfinite(lam) || !std::isfinite(nu))
    return fail(c, CVBA_ERR_INVALID_ARG, "set_damping: need lambda > 0 and nu >= 1");
  DeviceGuard g(c->device);
  CK(h2d(c, &c->d.ctrl->lam, &lam, sizeof(double)), "set lambda");
  CK(h2d(c, &c->d.ctrl->nu, &nu, sizeof(double)), "set nu");
  return CVBA_OK;
}

namespace {
// Checkpoint buffer: header, then poses (K x 12) and landmarks (M x 3, caller order).
struct StateHeader {
  char magic[8];        // "CVBASTA1"
  int32_t K, M, N, fixed_kf;
  double lam, nu;
};
constexpr char kStateMagic[8] = {'C', 'V', 'B', 'A', 'S', 'T', 'A', '1'};
size_t state_bytes(const cvba_ctx* c) {
  return sizeof(StateHeader) + sizeof(double) * ((size_t)c->K * 12 + (size_t)c->M * 3);
}
}  // namespace

cvba_status cvba_get_state(cvba_ctx* c, void* buf, size_t* bytes) {
  if (!c || !bytes) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "get_state: set_observations first");
  const size_t need = state_bytes(c);
  if (!buf) {
    *bytes = need;
    return CVBA_OK;
  }
  if (*bytes < need) return fail(c, CVBA_ERR_INVALID_ARG, "get_state: buffer too small");
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, sizeof(h.magic));
  h.K = c->K, h.M = c->M, h.N = c->N, h.fixed_kf = c->fixed_kf;
  cvba_status st = cvba_get_damping(c, &h.lam, &h.nu);
  unsigned char* out = static_cast<unsigned char*>(buf);
  double* poses = reinterpret_cast<double*>(out + sizeof(StateHeader));
  std::vector<double> P((size_t)c->K * 12), L((size_t)c->M * 3);
  if (st == CVBA_OK) st = cvba_get_poses(c, P.data());
  if (st == CVBA_OK) st = cvba_get_landmarks(c, L.data());
  if (st != CVBA_OK) return st;
  std::memcpy(out, &h, sizeof(h));
  std::memcpy(poses, P.data(), P.size() * sizeof(double));
  std::memcpy(poses + P.size(), L.data(), L.size() * sizeof(double));
  *bytes = need;
  return CVBA_OK;
}

cvba_status cvba_set_state(cvba_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "set_state: set_observations first");
  if (bytes < sizeof(StateHeader)) return fail(c, CVBA_ERR_INVALID_ARG, "set_state: buffer too small");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, sizeof(h.magic)) != 0)
    return fail(c, CVBA_ERR_INVALID_ARG, "set_state: not a checkpoint of this library");
  if (h.K != c->K || h.M != c->M || h.N != c->N || h.fixed_kf != c->fixed_kf || bytes < state_bytes(c))
    return fail(c, CVBA_ERR_INVALID_ARG, "set_state: checkpoint of a different problem");
  std::vector<double> P((size_t)c->K * 12), L((size_t)c->M * 3);
  const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof(StateHeader);
  std::memcpy(P.data(), in, P.size() * sizeof(double));
  std::memcpy(L.data(), in + P.size() * sizeof(double), L.size() * sizeof(double));
  cvba_status st = cvba_set_poses(c, c->K, P.data(), c->fixed_kf);
  if (st == CVBA_OK) st = cvba_set_landmarks(c, c->M, L.data());
  if (st == CVBA_OK) st = cvba_set_damping(c, h.lam, h.nu);
  return st;
}

cvba_status cvba_get_layout(cvba_ctx* c, int32_t* lm_order, int32_t* obs_order, int32_t* lm_off) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (!c->have_layout) return fail(c, CVBA_ERR_STATE, "get_layout: no layout");
  if (lm_order) std::copy(c->lm_order.begin(), c->lm_order.end(), lm_order);
  if (obs_order) std::copy(c->obs_order.begin(), c->obs_order.end(), obs_order);
  if (lm_off) std::copy(c->lm_off.begin(), c->lm_off.end(), lm_off);
  return CVBA_OK;
}

cvba_status cvba_get_sizes(cvba_ctx* c, int* n_kf, int* n_cams, int* n_lm, int* n_obs, int* n_pairs) {
  if (!c) return CVBA_ERR_INVALID_ARG;
  if (n_kf) *n_kf = c->K;
  if (n_cams) *n_cams = c->C;
  if (n_lm) *n_lm = c->M;
  if (n_obs) *n_obs = c->N;
  if (n_pairs) *n_pairs = c->have_layout ? c->P : 0;
  return CVBA_OK;
}

cvba_status cvba_solve_launch_count(cvba_ctx* c, int iters, int* n) {
  if (!c || !n || iters < 0) return CVBA_ERR_INVALID_ARG;
  *n = iters > 0 ? kernels_per_solve_init() + iters * (c->have_layout ? solve_kernels_per_iteration(c->d)
                                                                    : kernels_per_iteration()) : 0;
  return CVBA_OK;
}

}  // extern "C"

// ============================================================== batched windows

struct cvba_batch {
  std::vector<cvba_ctx*> ctxs;
  int device = 0;
  cudaStream_t stream = nullptr;
  int mixed = 0;
  int chol_cs = 4;
  void* dbuf = nullptr;              // Dev array and work lists
  size_t dbuf_bytes = 0;
  std::vector<Dev> host_devs, fallback;
  BatchLaunch L;
  cudaGraphExec_t graph = nullptr;
  cvba_ctx::Key key;
  int key_cs = 0;
  std::vector<Dev> snap;             // views the plan was built from
  std::string err;
};

namespace {

cvba_status bfail(cvba_batch* b, cvba_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

void batch_drop_graph(cvba_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->key = cvba_ctx::Key{};
}

cvba_status ensure_trace(cvba_ctx* c, int iters) {
  if (iters <= c->trace_cap) return CVBA_OK;
  CK(cudaStreamSynchronize(c->stream), "sync");
  if (c->d_trace) cudaFree(c->d_trace);
  c->d_trace = nullptr;
  c->trace_cap = 0;
  CK(cudaMalloc(&c->d_trace, sizeof(cvba_iter) * (size_t)iters), "alloc trace");
  c->trace_cap = iters;
  c->d.trace = c->d_trace;
  return CVBA_OK;
}

// (Re)build the device plan and capture the graph of `o->iters` batched iterations.
cvba_status batch_prepare(cvba_batch* b, const cvba_opts* o) {
  const int n = (int)b->ctxs.size();
  for (cvba_ctx* c : b->ctxs) {
    if (!c->have_layout) return bfail(b, CVBA_ERR_STATE, "batch: every window needs set_observations");
    cvba_status st = ensure_trace(c, o->iters);
    if (st != CVBA_OK) return bfail(b, st, c->err);
    c->d.trace = c->d_trace;
  }
  bool same = (int)b->snap.size() == n && b->graph && b->key_cs == b->chol_cs;
  for (int w = 0; same && w < n; ++w) same = std::memcmp(&b->snap[w], &b->ctxs[w]->d, sizeof(Dev)) == 0;
  const cvba_ctx::Key key = make_key(o, b->mixed != 0);
  if (same && key == b->key) return CVBA_OK;
  batch_drop_graph(b);
  // views, plan sizes, work lists
  b->snap.clear();
  b->host_devs.clear();
  for (cvba_ctx* c : b->ctxs) {
    b->snap.push_back(c->d);
    b->host_devs.push_back(c->d);
  }
  BatchLaunch& L = b->L;
  L = BatchLaunch{};
  L.n_win = n;
  L.mixed = b->mixed;
  L.chol_cs = b->chol_cs;
  batch_plan_sizes(b->host_devs.data(), n, L);
  b->fallback.clear();
  std::vector<int2> lin, kf, sch, blk, dir, win;
  for (int w = 0; w < n; ++w) {
    const Dev& d = b->host_devs[w];
    if (d.chol_fallback) b->fallback.push_back(d);
    for (int t = 0; t < d.n_lin_tiles; ++t) lin.push_back(make_int2(w, t));
    for (int a = 0; a < d.K; ++a) kf.push_back(make_int2(w, a));
    for (int t = 0; t < d.n_schur_tiles; ++t) sch.push_back(make_int2(w, t));
    for (int32_t t : b->ctxs[w]->act_blk) blk.push_back(make_int2(w, t));
    for (int t = 0; t < d.n_direct_tiles; ++t) dir.push_back(make_int2(w, t));
    win.push_back(make_int2(w, 0));
  }
  const size_t n_items = lin.size() + kf.size() + sch.size() + blk.size() + dir.size() + win.size();
  const size_t bytes = sizeof(Dev) * n + sizeof(int2) * n_items + 256;
  cvba_ctx* c = b->ctxs[0];
  if (bytes > b->dbuf_bytes) {
    if (b->dbuf) cudaFree(b->dbuf);
    b->dbuf = nullptr;
    b->dbuf_bytes = 0;
    CK(cudaMalloc(&b->dbuf, bytes), "alloc batch plan");
    b->dbuf_bytes = bytes;
  }
  std::vector<unsigned char> h(bytes, 0);
  std::memcpy(h.data(), b->host_devs.data(), sizeof(Dev) * n);
  size_t off = sizeof(Dev) * n;
  off = (off + 15) / 16 * 16;
  auto put = [&](const std::vector<int2>& v, const int2** dst, int* cnt) {
    *dst = reinterpret_cast<const int2*>(static_cast<unsigned char*>(b->dbuf) + off);
    *cnt = (int)v.size();
    if (!v.empty()) std::memcpy(h.data() + off, v.data(), v.size() * sizeof(int2));
    off += v.size() * sizeof(int2);
  };
  L.wins = static_cast<const Dev*>(b->dbuf);
  int n_win_items = 0;
  put(lin, &L.lin_items, &L.n_lin);
  put(kf, &L.kf_items, &L.n_kf);
  put(sch, &L.schur_items, &L.n_schur);
  put(blk, &L.blk_items, &L.n_blkit);
  put(dir, &L.direct_items, &L.n_direct);
  put(win, &L.win_items, &n_win_items);
  L.fallback_host = b->fallback.data();
  CK(cudaMemcpy(b->dbuf, h.data(), bytes, cudaMemcpyHostToDevice), "upload batch plan");
  // capture
  cudaGraph_t gr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = enqueue_batch_init(L, o->lambda0, o->huber_delta, o->z_min, o->iters, key.reset, key.refine,
                                     b->stream);
  for (int it = 0; it < o->iters && e == cudaSuccess; ++it) e = enqueue_batch_iteration(L, b->stream);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &gr);
  if (e != cudaSuccess) return cuda_fail(c, e, "enqueue batch");
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
  e = cudaGraphInstantiate(&b->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(c, e, "instantiate batch graph");
  b->key = key;
  b->key_cs = b->chol_cs;
  return CVBA_OK;
}

}  // namespace

extern "C" {

cvba_status cvba_batch_create(cvba_batch** out, int n_win, cvba_ctx* const* ctxs) {
  if (!out || n_win < 1 || !ctxs) return CVBA_ERR_INVALID_ARG;
  *out = nullptr;
  for (int w = 0; w < n_win; ++w) {
    if (!ctxs[w]) return CVBA_ERR_INVALID_ARG;
    if (ctxs[w]->device != ctxs[0]->device || ctxs[w]->prec != ctxs[0]->prec) return CVBA_ERR_INVALID_ARG;
  }
  cvba_batch* b = new cvba_batch();
  b->ctxs.assign(ctxs, ctxs + n_win);
  b->device = ctxs[0]->device;
  b->stream = ctxs[0]->stream;
  b->mixed = ctxs[0]->prec == CVBA_MIXED ? 1 : 0;
  *out = b;
  return CVBA_OK;
}

void cvba_batch_destroy(cvba_batch* b) {
  if (!b) return;
  {
    DeviceGuard g(b->device);
    cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    if (b->dbuf) cudaFree(b->dbuf);
  }
  delete b;
}

const char* cvba_batch_last_error(const cvba_batch* b) { return b ? b->err.c_str() : ""; }

cvba_status cvba_batch_set_chol_cluster(cvba_batch* b, int cs) {
  if (!b || !(cs == 2 || cs == 4 || cs == 8 || cs == 16)) return CVBA_ERR_INVALID_ARG;
  b->chol_cs = cs;
  return CVBA_OK;
}

cvba_status cvba_batch_solve_async(cvba_batch* b, const cvba_opts* o) {
  if (!b || !o) return CVBA_ERR_INVALID_ARG;
  if (!opts_ok(o)) return bfail(b, CVBA_ERR_INVALID_ARG, "batch solve: bad options");
  if (o->iters == 0) return CVBA_OK;
  DeviceGuard g(b->device);
  cvba_status st = batch_prepare(b, o);
  if (st != CVBA_OK) {
    if (b->err.empty()) b->err = b->ctxs[0]->err;
    return st;
  }
  if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, CVBA_ERR_CUDA, "batch graph launch failed");
  }
  return CVBA_OK;
}

cvba_status cvba_batch_solve(cvba_batch* b, const cvba_opts* o, cvba_iter* traces) {
  cvba_status st = cvba_batch_solve_async(b, o);
  if (st != CVBA_OK || o->iters == 0) return st;
  DeviceGuard g(b->device);
  if (traces) {
    for (size_t w = 0; w < b->ctxs.size(); ++w)
      if (cudaMemcpyAsync(traces + w * (size_t)o->iters, b->ctxs[w]->d_trace, sizeof(cvba_iter) * (size_t)o->iters,
                          cudaMemcpyDeviceToHost, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, CVBA_ERR_CUDA, "batch trace copy failed");
      }
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, CVBA_ERR_CUDA, "batch solve failed");
  }
  return CVBA_OK;
}

cvba_status cvba_batch_launch_count(cvba_batch* b, const cvba_opts* o, int* n) {
  if (!b || !o || !n) return CVBA_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  cvba_status st = batch_prepare(b, o);
  if (st != CVBA_OK) return st;
  *n = o->iters > 0 ? 1 + o->iters * batch_kernels_per_iteration(b->L) : 0;
  return CVBA_OK;
}

namespace {
// Autotune results, per device and batch configuration: the device (name, SM count, compute
// capability) and every window's shape (keyframes, cameras, landmarks, observations, pairs)
// with the precision.  Process-wide; guarded by a mutex.
struct TuneKey {
  std::string device;
  std::vector<int64_t> shape;
  bool operator<(const TuneKey& o) const { return device != o.device ? device < o.device : shape < o.shape; }
};
struct TuneValue {
  int lin, schur, cs;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneValue> g_tune_cache;

TuneKey tune_key(const cvba_batch* b) {
  TuneKey k;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) cudaGetLastError();
  k.device = std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "/" +
             std::to_string(prop.major) + "." + std::to_string(prop.minor);
  k.shape.push_back(b->mixed);
  for (const cvba_ctx* c : b->ctxs)
    for (int64_t v : {(int64_t)c->K, (int64_t)c->C, (int64_t)c->M, (int64_t)c->N, (int64_t)c->P}) k.shape.push_back(v);
  return k;
}
}  // namespace

extern "C" void cvba_batch_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache.clear();
}

// Autotuner: times a 2-iteration batched solve for each candidate (lin tile pairs, Schur
// tile landmarks), then each Cholesky cluster size, keeps the fastest and restores every
// window's state.  The choice is cached per device and batch configuration: a later call
// with the same configuration applies it without timing.  Writes the chosen values (any
// pointer may be NULL).
cvba_status cvba_batch_autotune(cvba_batch* b, const cvba_opts* o, int* best_lin, int* best_schur, int* best_cs) {
  if (!b || !o) return CVBA_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  const int n = (int)b->ctxs.size();
  const TuneKey key = tune_key(b);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const TuneValue v = it->second;
      for (int w = 0; w < n; ++w) {
        const cvba_status st = cvba_set_tuning(b->ctxs[w], v.lin, v.schur);
        if (st != CVBA_OK) return bfail(b, st, b->ctxs[w]->err);
      }
      b->chol_cs = v.cs;
      if (best_lin) *best_lin = v.lin;
      if (best_schur) *best_schur = v.schur;
      if (best_cs) *best_cs = v.cs;
      return CVBA_OK;
    }
  }
  std::vector<std::vector<double>> P(n), Lm(n);
  std::vector<double> lam(n), nu(n);
  for (int w = 0; w < n; ++w) {
    cvba_ctx* c = b->ctxs[w];
    P[w].resize((size_t)c->K * 12);
    Lm[w].resize((size_t)c->M * 3);
    if (cvba_get_poses(c, P[w].data()) != CVBA_OK || cvba_get_landmarks(c, Lm[w].data()) != CVBA_OK ||
        cvba_get_damping(c, &lam[w], &nu[w]) != CVBA_OK)
      return bfail(b, CVBA_ERR_STATE, "autotune: windows need a layout");
  }
  auto restore = [&]() -> cvba_status {
    for (int w = 0; w < n; ++w) {
      cvba_ctx* c = b->ctxs[w];
      cvba_status st = cvba_set_poses(c, c->K, P[w].data(), c->fixed_kf);
      if (st == CVBA_OK) st = cvba_set_landmarks(c, c->M, Lm[w].data());
      if (st == CVBA_OK) st = cvba_set_damping(c, lam[w], nu[w]);
      if (st != CVBA_OK) return st;
    }
    return CVBA_OK;
  };
  cvba_opts t = *o;
  t.iters = 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](float* ms) -> cvba_status {
    cvba_status st = cvba_batch_solve(b, &t, nullptr);             // prepares + warms the graph
    if (st == CVBA_OK) st = restore();
    if (st != CVBA_OK) return st;
    cudaEventRecord(e0, b->stream);
    st = cvba_batch_solve_async(b, &t);
    cudaEventRecord(e1, b->stream);
    if (st == CVBA_OK && cudaEventSynchronize(e1) != cudaSuccess) st = CVBA_ERR_CUDA;
    if (st == CVBA_OK) cudaEventElapsedTime(ms, e0, e1);
    cvba_status st2 = restore();
    return st != CVBA_OK ? st : st2;
  };
  const int lin_c[] = {32, 64, 128, 256};
  const int sch_c[] = {8, 16, 32, 64, 128};
  float best = 1e30f;
  int bl = 0, bs = 0, bc = b->chol_cs;
  cvba_status st = CVBA_OK;
  for (int li : lin_c) {
    for (int sc : sch_c) {
      for (int w = 0; w < n && st == CVBA_OK; ++w) st = cvba_set_tuning(b->ctxs[w], li, sc);
      float ms = 0.f;
      if (st == CVBA_OK) st = timed(&ms);
      if (st != CVBA_OK) break;
      if (ms < best) {
        best = ms;
        bl = li;
        bs = sc;
      }
    }
    if (st != CVBA_OK) break;
  }
  if (st == CVBA_OK)
    for (int w = 0; w < n && st == CVBA_OK; ++w) st = cvba_set_tuning(b->ctxs[w], bl, bs);
  if (st == CVBA_OK) {
    best = 1e30f;
    for (int cs : {2, 4, 8, 16}) {
      b->chol_cs = cs;
      float ms = 0.f;
      st = timed(&ms);
      if (st != CVBA_OK) break;
      if (ms < best) {
        best = ms;
        bc = cs;
      }
    }
    b->chol_cs = bc;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CVBA_OK) return bfail(b, st, "autotune failed: " + b->ctxs[0]->err);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = TuneValue{bl, bs, bc};
  }
  if (best_lin) *best_lin = bl;
  if (best_schur) *best_schur = bs;
  if (best_cs) *best_cs = bc;
  return CVBA_OK;
}

}  // extern "C"
