// Host part of a window's device layout: the landmark order, the observation order and the
// (landmark, keyframe) pairs, computed in parallel on the host cores.
//
// Definition (what the solve's kernels rely on, and what the layout tests check exactly):
//  - internal landmarks are the caller's ordered by (first observing keyframe, last observing
//    keyframe, caller index);
//  - observation slots are ordered by (internal landmark, keyframe, camera, caller index);
//  - pairs are the distinct (internal landmark, keyframe) runs of the slots, in slot order.
//
// Algorithm: the caller's landmarks are cut into buckets of 2^s consecutive indices (8k to
// 16k observations a bucket on average); every observation becomes a 64-bit key (landmark
// within its bucket, keyframe, camera, caller index); a parallel counting pass and stable
// scatter group the keys by bucket; each bucket, in a core's cache, is then put in order by
// two stable counting sorts, by (keyframe, camera) and then by landmark, which leaves every
// landmark's keys in (keyframe, camera, caller index) order; the landmarks are ordered by a
// stable counting sort on the first keyframe and, within each first keyframe, one on the
// last; and the slots and pairs are filled group by group from the keys, with no gather of
// the caller's arrays.  Every step is deterministic and independent
// of the thread count and of which thread takes which bucket.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cvba_internal.h"

namespace cvba {

int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h == 0 ? 1u : h, 32u));
}

namespace {

// Worker threads kept for the library's lifetime, so a parallel section costs a wake-up
// rather than thread creation (a layout runs about ten sections).  One section runs on the
// pool at a time; a section started while another holds the pool, or from inside a task,
// runs on threads of its own (the previous scheme), so nesting and concurrent contexts cannot
// deadlock.  Workers are detached and never joined: they sleep on the condition variable.
thread_local bool tl_pool_worker = false;
thread_local bool tl_in_section = false;             // this thread runs a pool section's task 0

class Pool {
 public:
  static Pool& get() {
    static Pool* p = new Pool();                    // never destroyed (detached workers)
    return *p;
  }
  // Runs fn(0..n-1); false (nothing run) if the pool is busy or the caller is a worker.
  bool run(int n, const std::function<void(int)>& fn) {
    if (tl_pool_worker || tl_in_section) return false;   // nested: never re-lock run_mu_
    std::unique_lock<std::mutex> section(run_mu_, std::try_to_lock);
    if (!section.owns_lock()) return false;
    uint64_t g;
    {
      std::lock_guard<std::mutex> lk(mu_);
      while ((int)n_workers_ < n - 1) {
        std::thread(&Pool::worker, this).detach();
        ++n_workers_;
      }
      fn_ = &fn;
      n_ = n;
      next_ = 1;
      remaining_ = n - 1;
      g = ++gen_;
    }
    cv_.notify_all();
    tl_in_section = true;
    fn(0);
    help(g);
    tl_in_section = false;
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return remaining_ == 0; });
    fn_ = nullptr;
    return true;
  }

 private:
  // Take tasks of generation g until none is left; a task index is handed out under the
  // lock together with the generation check, so a late worker never runs a task of a
  // section that has ended, and the section's caller waits until every taken task is done.
  void help(uint64_t g) {
    for (;;) {
      const std::function<void(int)>* f;
      int t;
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (gen_ != g || fn_ == nullptr || next_ >= n_) return;
        f = fn_;
        t = next_++;
      }
      (*f)(t);
      std::lock_guard<std::mutex> lk(mu_);
      if (--remaining_ == 0) done_cv_.notify_all();
    }
  }
  void worker() {
    tl_pool_worker = true;
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
      }
      help(seen);
    }
  }
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* fn_ = nullptr;
  int n_ = 0, next_ = 0, remaining_ = 0;
  unsigned n_workers_ = 0;
  uint64_t gen_ = 0;
};

}  // namespace

void parallel_tasks(int n, const std::function<void(int)>& fn) {
  if (n <= 1) {
    if (n == 1) fn(0);
    return;
  }
  if (Pool::get().run(n, fn)) return;
  std::vector<std::thread> pool;
  pool.reserve(n - 1);
  for (int t = 1; t < n; ++t) pool.emplace_back(fn, t);
  fn(0);
  for (auto& th : pool) th.join();
}

void parallel_for(int64_t n, int threads, const std::function<void(int64_t, int64_t, int)>& fn) {
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, n / 4096 + 1));
  if (threads == 1) {
    fn(0, n, 0);
    return;
  }
  parallel_tasks(threads, [&](int t) { fn(n * t / threads, n * (t + 1) / threads, t); });
}

void parallel_ranges(int64_t n, const std::function<void(int64_t, int64_t, int)>& fn) {
  const int threads = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n));
  if (threads == 1) {
    fn(0, n, 0);
    return;
  }
  parallel_tasks(threads, [&](int t) { fn(n * t / threads, n * (t + 1) / threads, t); });
}

bool compute_host_layout(int K, int C, int M, int N, int fixed_kf, const int32_t* kf, const int32_t* cam,
                         const int32_t* lm, HostLayout& L, std::string& err) {
  static_assert(K_MAX <= 256 && C_MAX <= 256, "keyframe and camera take 8 bits of a sort key");
  const int T = host_threads();
  // work arrays live in L (kept between calls, so a window of the same size reuses them
  // without new pages)
  std::vector<uint64_t>& rec = L.rec_key;
  std::vector<uint64_t>& grp = L.grp;
  std::vector<int64_t>& goff = L.goff;
  // Landmark buckets: 2^sh consecutive caller landmarks each, sized so that a bucket holds
  // 8k to 16k observations on average (its keys and a copy stay in a core's cache) and at most
  // 2^16 landmarks.
  int sh = 0;
  while (sh < 16 && ((int64_t)N << (sh + 1)) <= (int64_t)16384 * std::max(M, 1)) ++sh;
  const int W = 1 << sh;
  const int B = std::max(1, (int)(((int64_t)M + W - 1) >> sh));
  // Every observation as a 64-bit sort key: its landmark's index within the bucket in bits
  // 48..63, keyframe in 40..47, camera in 32..39, caller index below.  Ordering a bucket's
  // keys orders it by (landmark, keyframe, camera, caller index), and keyframe, camera and
  // caller index come back out of the key by shifts, without a gather.
  auto key_of = [&](int64_t n) {
    return ((uint64_t)(uint32_t)(lm[n] & (W - 1)) << 48) | ((uint64_t)(uint32_t)kf[n] << 40) |
           ((uint64_t)(uint32_t)cam[n] << 32) | (uint32_t)n;
  };
  auto kf_of = [](uint64_t key) { return (int32_t)((key >> 40) & 0xff); };
  auto cam_of = [](uint64_t key) { return (int32_t)((key >> 32) & 0xff); };
  // --- group by bucket: parallel counting pass and stable scatter (chunks of the caller's
  //     order, so each bucket receives its keys in caller order)
  std::vector<int64_t> cnt((size_t)T * B, 0);          // [chunk][bucket]
  std::vector<int64_t> kf_cnt((size_t)T * K, 0);       // [chunk][keyframe]
  parallel_tasks(T, [&](int c) {
    const int64_t n0 = (int64_t)N * c / T, n1 = (int64_t)N * (c + 1) / T;
    int64_t* cc = cnt.data() + (size_t)c * B;
    int64_t* kc = kf_cnt.data() + (size_t)c * K;
    for (int64_t n = n0; n < n1; ++n) {
      cc[lm[n] >> sh]++;
      kc[kf[n]]++;
    }
  });
  std::vector<int64_t> boff((size_t)B + 1, 0);
  {
    int64_t acc = 0;                                   // cnt becomes each chunk's write position
    for (int b = 0; b < B; ++b) {
      boff[b] = acc;
      for (int c = 0; c < T; ++c) {
        const int64_t m = cnt[(size_t)c * B + b];
        cnt[(size_t)c * B + b] = acc;
        acc += m;
      }
    }
    boff[B] = acc;
  }
  rec.resize((size_t)N);
  parallel_tasks(T, [&](int c) {
    const int64_t n0 = (int64_t)N * c / T, n1 = (int64_t)N * (c + 1) / T;
    int64_t* p = cnt.data() + (size_t)c * B;
    for (int64_t n = n0; n < n1; ++n) rec[p[lm[n] >> sh]++] = key_of(n);
  });
  // --- per bucket, in cache: a stable counting sort by (keyframe, camera), then a stable
  //     one by landmark, which leaves each landmark's keys in (keyframe, camera, caller
  //     index) order; then each landmark's first and last keyframe and its pair count
  goff.resize((size_t)M + 1);
  grp.resize((size_t)N);
  std::vector<int32_t>& first = L.first;           // every entry is written below
  std::vector<int32_t>& last = L.last;
  std::vector<int32_t>& npair_of = L.npair_of;
  first.resize((size_t)M);
  last.resize((size_t)M);
  npair_of.resize((size_t)M);
  {
    const int KC = K * C;
    std::atomic<int> next_bucket{0};
    parallel_tasks(T, [&](int) {
      thread_local std::vector<uint64_t> tmp;      // per thread, kept by the pool's workers
      thread_local std::vector<int64_t> h;
      if (h.size() < (size_t)std::max(KC, W) + 1) h.resize((size_t)std::max(KC, W) + 1);
      for (int b; (b = next_bucket.fetch_add(1)) < B;) {
        const int64_t e0 = boff[b], E = boff[b + 1] - e0;
        const int lo = b << sh, nl = std::min(M - lo, W);
        const uint64_t* src = rec.data() + e0;
        if ((int64_t)tmp.size() < E) tmp.resize((size_t)E);
        std::fill(h.begin(), h.begin() + KC + 1, 0);
        for (int64_t a = 0; a < E; ++a) h[(size_t)kf_of(src[a]) * C + cam_of(src[a]) + 1]++;
        for (int d = 0; d < KC; ++d) h[d + 1] += h[d];
        for (int64_t a = 0; a < E; ++a) tmp[h[(size_t)kf_of(src[a]) * C + cam_of(src[a])]++] = src[a];
        std::fill(h.begin(), h.begin() + nl + 1, 0);
        for (int64_t a = 0; a < E; ++a) h[(tmp[a] >> 48) + 1]++;
        for (int j = 0; j < nl; ++j) h[j + 1] += h[j];
        for (int j = 0; j < nl; ++j) goff[lo + j] = e0 + h[j];
        uint64_t* dst = grp.data() + e0;
        for (int64_t a = 0; a < E; ++a) dst[h[tmp[a] >> 48]++] = tmp[a];
        for (int j = 0; j < nl; ++j) {                 // h[j] is now the end of landmark lo + j
          const int64_t g0 = j == 0 ? 0 : h[j - 1], m = h[j] - g0;
          const uint64_t* g = dst + g0;
          first[lo + j] = m > 0 ? kf_of(g[0]) : K;
          last[lo + j] = m > 0 ? kf_of(g[m - 1]) : -1;
          int np = 0;                                  // distinct keyframes: the landmark's pairs
          for (int64_t q = 0; q < m; ++q)
            if (q == 0 || kf_of(g[q]) != kf_of(g[q - 1])) ++np;
          npair_of[lo + j] = np;
        }
      }
    });
  }
  goff[M] = N;
  for (int j = 0; j < M; ++j)
    if (goff[j + 1] - goff[j] < 2) {
      err = "landmark " + std::to_string(j) + " has fewer than 2 observations";
      return false;
    }
  for (int a = 0; a < K; ++a) {
    int64_t n_a = 0;
    for (int c = 0; c < T; ++c) n_a += kf_cnt[(size_t)c * K + a];
    if (a != fixed_kf && n_a == 0) {
      err = "keyframe " + std::to_string(a) + " is free but has no observations";
      return false;
    }
  }
  // --- landmark order (first, last, caller index): a parallel stable counting sort by first
  //     keyframe (every landmark has an observation, so first and last are keyframes), then
  //     per first keyframe a stable counting sort by last; each landmark's slot and pair
  //     counts are placed at its rank on the way, and summed into offsets after
  L.lm_order.resize(M);
  L.lm_rank.resize(M);
  L.lm_off.resize((size_t)M + 1);
  L.lm_pair.resize((size_t)M + 1);
  {
    std::vector<int64_t> fpos((size_t)T * K, 0);       // [chunk][first]
    std::vector<int64_t> foff((size_t)K + 1, 0);
    std::vector<int32_t>& by_first = L.by_first;    // every entry is written below
    by_first.resize((size_t)M);
    parallel_tasks(T, [&](int c) {
      const int64_t j0 = (int64_t)M * c / T, j1 = (int64_t)M * (c + 1) / T;
      int64_t* fc = fpos.data() + (size_t)c * K;
      for (int64_t j = j0; j < j1; ++j) fc[first[j]]++;
    });
    {
      int64_t acc = 0;
      for (int f = 0; f < K; ++f) {
        foff[f] = acc;
        for (int c = 0; c < T; ++c) {
          const int64_t m = fpos[(size_t)c * K + f];
          fpos[(size_t)c * K + f] = acc;
          acc += m;
        }
      }
      foff[K] = acc;
    }
    parallel_tasks(T, [&](int c) {
      const int64_t j0 = (int64_t)M * c / T, j1 = (int64_t)M * (c + 1) / T;
      int64_t* fc = fpos.data() + (size_t)c * K;
      for (int64_t j = j0; j < j1; ++j) by_first[fc[first[j]]++] = (int32_t)j;
    });
    std::atomic<int> next_first{0};
    parallel_tasks(T, [&](int) {
      std::vector<int64_t> h((size_t)K + 1);
      for (int f; (f = next_first.fetch_add(1)) < K;) {
        const int64_t i0 = foff[f], i1 = foff[f + 1];
        std::fill(h.begin(), h.end(), 0);
        for (int64_t i = i0; i < i1; ++i) h[last[by_first[i]] + 1]++;
        h[0] = i0;
        for (int k = 0; k < K; ++k) h[k + 1] += h[k];
        for (int64_t i = i0; i < i1; ++i) {
          const int j = by_first[i];
          const int64_t r = h[last[j]]++;
          L.lm_order[r] = j;
          L.lm_rank[j] = (int32_t)r;
          L.lm_off[r + 1] = (int32_t)(goff[j + 1] - goff[j]);
          L.lm_pair[r + 1] = npair_of[j];
        }
      }
    });
    // offsets: per-chunk sums, then each chunk's running sums from its base
    std::vector<int64_t> so((size_t)T + 1, 0), sp((size_t)T + 1, 0);
    parallel_tasks(T, [&](int c) {
      const int64_t i0 = (int64_t)M * c / T, i1 = (int64_t)M * (c + 1) / T;
      int64_t a = 0, q = 0;
      for (int64_t i = i0; i < i1; ++i) {
        a += L.lm_off[i + 1];
        q += L.lm_pair[i + 1];
      }
      so[c + 1] = a;
      sp[c + 1] = q;
    });
    for (int c = 0; c < T; ++c) {
      so[c + 1] += so[c];
      sp[c + 1] += sp[c];
    }
    L.lm_off[0] = 0;
    L.lm_pair[0] = 0;
    parallel_tasks(T, [&](int c) {
      const int64_t i0 = (int64_t)M * c / T, i1 = (int64_t)M * (c + 1) / T;
      int64_t a = so[c], q = sp[c];
      for (int64_t i = i0; i < i1; ++i) {
        a += L.lm_off[i + 1];
        q += L.lm_pair[i + 1];
        L.lm_off[i + 1] = (int32_t)a;
        L.lm_pair[i + 1] = (int32_t)q;
      }
    });
  }
  // --- slots: groups in internal order; distinct keyframe runs are the pairs
  const int P = L.lm_pair[M];
  L.obs_order.resize(N);
  L.obs_cam.resize(N);
  L.pair_kf.resize(P);
  L.pair_lm.resize(P);
  L.pair_obs.resize((size_t)P + 1);
  parallel_for(M, T, [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i) {
      if (i + 8 < i1) __builtin_prefetch(grp.data() + goff[L.lm_order[i + 8]]);   // groups are met in rank order
      const uint64_t* g = grp.data() + goff[L.lm_order[i]];
      const int64_t m = L.lm_off[i + 1] - L.lm_off[i];
      const int64_t s0 = L.lm_off[i];
      int q = L.lm_pair[i];
      for (int64_t a = 0; a < m; ++a) {
        const int32_t k = kf_of(g[a]);
        L.obs_order[s0 + a] = (int32_t)(uint32_t)g[a];
        L.obs_cam[s0 + a] = cam_of(g[a]);
        if (a == 0 || k != kf_of(g[a - 1])) {
          L.pair_kf[q] = k;
          L.pair_lm[q] = (int32_t)i;
          L.pair_obs[q] = (int32_t)(s0 + a);
          ++q;
        }
      }
    }
  });
  L.pair_obs[P] = N;
  return true;
}

}  // namespace cvba
