// Host part of a window's device layout: the landmark order, the observation order and the
// (landmark, keyframe) pairs, computed in parallel on the host cores.
//
// Definition (what the solve's kernels rely on, and what the layout tests check exactly):
//  - internal landmarks are the caller's ordered by (first observing keyframe, last observing
//    keyframe, caller index);
//  - observation slots are ordered by (internal landmark, keyframe, camera, caller index);
//  - pairs are the distinct (internal landmark, keyframe) runs of the slots, in slot order.
//
// Algorithm: every observation becomes a 64-bit key (keyframe * C + camera, caller index);
// the keys are grouped by the caller's landmark index with a parallel two-level counting
// sort (a radix pass into one landmark range per thread, then a counting sort inside each
// range); each landmark's keys are sorted in place (insertion sort: groups hold a few to a
// few tens of observations), which orders them by (keyframe, camera, caller index); the
// landmarks are ordered by two stable counting sorts; and the slots and pairs are filled group
// by group from the keys, with no gather of the caller's arrays.  Every step is
// deterministic and independent of the thread count.
#include <algorithm>
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

namespace {

// Stable counting sort of idx by key[idx] in [0, n_keys).
void counting_sort(std::vector<int32_t>& idx, const std::vector<int32_t>& key, int n_keys) {
  std::vector<int64_t> cnt((size_t)n_keys + 1, 0);
  for (int32_t i : idx) cnt[(size_t)key[i] + 1]++;
  for (int k = 0; k < n_keys; ++k) cnt[k + 1] += cnt[k];
  std::vector<int32_t> out(idx.size());
  for (int32_t i : idx) out[cnt[key[i]]++] = i;
  idx.swap(out);
}

}  // namespace

bool compute_host_layout(int K, int C, int M, int N, int fixed_kf, const int32_t* kf, const int32_t* cam,
                         const int32_t* lm, HostLayout& L, std::string& err) {
  const int T = host_threads();
  // work arrays live in L (kept between calls, so a window of the same size reuses them
  // without new pages)
  std::vector<int32_t>& rec_lm = L.rec_lm;
  std::vector<uint64_t>& rec_key = L.rec_key;
  std::vector<uint64_t>& grp = L.grp;
  std::vector<int64_t>& goff = L.goff;
  // Every observation as a 64-bit sort key: (keyframe * C + camera) above, caller index
  // below, so ordering the keys orders by (keyframe, camera, caller index), and the
  // keyframe and camera come back out of the key without a gather.
  auto key_of = [&](int64_t n) { return ((uint64_t)(uint32_t)(kf[n] * C + cam[n]) << 32) | (uint32_t)n; };
  // --- group by caller landmark: parallel radix pass (T landmark ranges), then a counting
  //     sort inside each range
  std::vector<int32_t> bucket_lo((size_t)T + 1);
  for (int b = 0; b <= T; ++b) bucket_lo[b] = (int32_t)((int64_t)M * b / T);
  std::vector<uint8_t> bucket_of((size_t)M);
  for (int b = 0; b < T; ++b)
    for (int j = bucket_lo[b]; j < bucket_lo[b + 1]; ++j) bucket_of[j] = (uint8_t)b;
  std::vector<int64_t> cnt((size_t)T * T, 0);          // [chunk][bucket]
  std::vector<int64_t> kf_cnt((size_t)T * K, 0);       // [chunk][keyframe]
  parallel_tasks(T, [&](int c) {
    const int64_t n0 = (int64_t)N * c / T, n1 = (int64_t)N * (c + 1) / T;
    int64_t* cc = cnt.data() + (size_t)c * T;
    int64_t* kc = kf_cnt.data() + (size_t)c * K;
    for (int64_t n = n0; n < n1; ++n) {
      cc[bucket_of[lm[n]]]++;
      kc[kf[n]]++;
    }
  });
  std::vector<int64_t> pos((size_t)T * T), boff((size_t)T + 1, 0);
  {
    int64_t acc = 0;
    for (int b = 0; b < T; ++b) {
      boff[b] = acc;
      for (int c = 0; c < T; ++c) {
        pos[(size_t)c * T + b] = acc;
        acc += cnt[(size_t)c * T + b];
      }
    }
    boff[T] = acc;
  }
  rec_lm.resize((size_t)N);
  rec_key.resize((size_t)N);
  parallel_tasks(T, [&](int c) {
    const int64_t n0 = (int64_t)N * c / T, n1 = (int64_t)N * (c + 1) / T;
    int64_t* p = pos.data() + (size_t)c * T;
    for (int64_t n = n0; n < n1; ++n) {
      const int b = bucket_of[lm[n]];
      const int64_t q = p[b]++;
      rec_lm[q] = lm[n];
      rec_key[q] = key_of(n);
    }
  });
  goff.resize((size_t)M + 1);
  grp.resize((size_t)N);
  parallel_tasks(T, [&](int b) {
    const int lo = bucket_lo[b], hi = bucket_lo[b + 1];
    std::vector<int64_t> fill((size_t)(hi - lo), 0);
    for (int64_t q = boff[b]; q < boff[b + 1]; ++q) fill[rec_lm[q] - lo]++;
    int64_t acc = boff[b];
    for (int j = lo; j < hi; ++j) {       // goff[j] for the range's own landmarks only
      const int64_t m = fill[j - lo];
      goff[j] = acc;
      fill[j - lo] = acc;
      acc += m;
    }
    for (int64_t q = boff[b]; q < boff[b + 1]; ++q) grp[fill[rec_lm[q] - lo]++] = rec_key[q];
  });
  goff[M] = N;
  // --- per landmark: sort its keys (stable order is kept by the caller index in the key),
  //     first / last keyframe
  std::vector<int32_t> first((size_t)M), last((size_t)M), npair_of((size_t)M);
  parallel_for(M, T, [&](int64_t j0, int64_t j1, int) {
    for (int64_t j = j0; j < j1; ++j) {
      uint64_t* g = grp.data() + goff[j];
      const int64_t m = goff[j + 1] - goff[j];
      for (int64_t a = 1; a < m; ++a) {
        const uint64_t v = g[a];
        int64_t b = a - 1;
        while (b >= 0 && g[b] > v) {
          g[b + 1] = g[b];
          --b;
        }
        g[b + 1] = v;
      }
      first[j] = m > 0 ? (int32_t)((g[0] >> 32) / C) : K;
      last[j] = m > 0 ? (int32_t)((g[m - 1] >> 32) / C) : -1;
      int np = 0;                                  // distinct keyframes: the landmark's pairs
      for (int64_t a = 0; a < m; ++a)
        if (a == 0 || (uint32_t)(g[a] >> 32) / C != (uint32_t)(g[a - 1] >> 32) / C) ++np;
      npair_of[j] = np;
    }
  });
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
  // --- landmark order: (first, last, caller index)
  L.lm_order.resize(M);
  for (int j = 0; j < M; ++j) L.lm_order[j] = j;
  counting_sort(L.lm_order, last, K);
  counting_sort(L.lm_order, first, K);
  L.lm_rank.resize(M);
  for (int i = 0; i < M; ++i) L.lm_rank[L.lm_order[i]] = i;
  // --- slots: groups in internal order; distinct keyframe runs are the pairs.  Offsets by
  //     prefix sums over the internal order, then one pass fills slots and pairs together.
  L.lm_off.resize((size_t)M + 1);
  L.lm_pair.resize((size_t)M + 1);
  {
    std::vector<int32_t> sz((size_t)M), np((size_t)M);
    parallel_for(M, T, [&](int64_t i0, int64_t i1, int) {
      for (int64_t i = i0; i < i1; ++i) {
        const int j = L.lm_order[i];
        sz[i] = (int32_t)(goff[j + 1] - goff[j]);
        np[i] = npair_of[j];
      }
    });
    L.lm_off[0] = 0;
    L.lm_pair[0] = 0;
    for (int i = 0; i < M; ++i) {
      L.lm_off[i + 1] = L.lm_off[i] + sz[i];
      L.lm_pair[i + 1] = L.lm_pair[i] + np[i];
    }
  }
  const int P = L.lm_pair[M];
  L.obs_order.resize(N);
  L.obs_cam.resize(N);
  L.pair_kf.resize(P);
  L.pair_lm.resize(P);
  L.pair_obs.resize((size_t)P + 1);
  parallel_for(M, T, [&](int64_t i0, int64_t i1, int) {
    for (int64_t i = i0; i < i1; ++i) {
      const uint64_t* g = grp.data() + goff[L.lm_order[i]];
      const int64_t m = L.lm_off[i + 1] - L.lm_off[i];
      const int64_t s0 = L.lm_off[i];
      int q = L.lm_pair[i];
      for (int64_t a = 0; a < m; ++a) {
        const uint32_t kc = (uint32_t)(g[a] >> 32);
        L.obs_order[s0 + a] = (int32_t)(uint32_t)g[a];
        L.obs_cam[s0 + a] = (int32_t)(kc % C);
        if (a == 0 || kc / C != (uint32_t)(g[a - 1] >> 32) / C) {
          L.pair_kf[q] = (int32_t)(kc / C);
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
