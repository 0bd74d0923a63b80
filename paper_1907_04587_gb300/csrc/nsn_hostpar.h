// nsn_hostpar.h -- host-side parallel passes of the layout build: a
// persistent pool of worker threads, a parallel exclusive scan and a stable
// counting sort whose results equal those of one sequential pass.  Plain
// C++17 (no CUDA), so that the CPU tests compile it on its own.
#pragma once
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include <sys/types.h>
#include <unistd.h>

namespace nsn {

// Host worker threads kept for the life of the process: a layout pass hands
// k = 1 .. n-1 to workers 1 .. n-1 and runs k = 0 itself.  Creating and
// joining a thread per pass cost tens of microseconds per thread, about ten
// times per rebuilt step.  One pass at a time (a mutex); a pass issued while
// another runs (another context's thread, or from inside a pass) runs its
// items on the calling thread.
class HostPool {
 public:
  static HostPool &get() {
    static HostPool pool;
    return pool;
  }
  // workers of this process (0 in a child forked after they started: they do
  // not exist there, and its passes run on the calling thread)
  int workers() const { return pid_ == getpid() ? int(th_.size()) : 0; }
  // false: the pool is busy, the caller runs the items itself
  bool run(int n, void (*call)(const void *, int), const void *obj) {
    std::unique_lock<std::mutex> busy(pass_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> g(m_);
      call_ = call; obj_ = obj; n_ = n; left_ = n - 1; ++gen_;
    }
    cv_.notify_all();
    call(obj, 0);
    std::unique_lock<std::mutex> g(m_);
    done_.wait(g, [&] { return left_ == 0; });
    return true;
  }
  ~HostPool() {
    if (pid_ != getpid()) {   // a forked child: the threads are not this process's
      for (std::thread &x : th_) x.detach();
      return;
    }
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread &x : th_) x.join();
  }

 private:
  HostPool() : pid_(getpid()) {
    const int hw = std::max(1, int(std::thread::hardware_concurrency()));
    const int nw = std::min(hw, 16) - 1;
    for (int w = 1; w <= nw; w++) th_.emplace_back([this, w] { loop(w); });
  }
  void loop(int w) {
    long seen = 0;
    for (;;) {
      void (*call)(const void *, int);
      const void *obj;
      {
        std::unique_lock<std::mutex> g(m_);
        cv_.wait(g, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        if (w >= n_) continue;
        call = call_; obj = obj_;
      }
      call(obj, w);
      std::lock_guard<std::mutex> g(m_);
      if (--left_ == 0) done_.notify_one();
    }
  }
  pid_t pid_;
  std::vector<std::thread> th_;
  std::mutex pass_, m_;
  std::condition_variable cv_, done_;
  void (*call_)(const void *, int) = nullptr;
  const void *obj_ = nullptr;
  int n_ = 0, left_ = 0;
  long gen_ = 0;
  bool stop_ = false;
};

// host threads for a layout pass over n items: one per ~64k items, at most
// the hardware threads and 16
inline int layout_threads(long long n) {
  const int hw = std::max(1, int(std::thread::hardware_concurrency()));
  return int(std::max(1LL, std::min<long long>({(n + 65535) / 65536, (long long)hw, 16LL})));
}

// Runs fn(k) for k = 0 .. n-1 (the calling thread takes k = 0) on the pool's
// workers; with more items than workers, or the pool busy, on the calling
// thread one after the other.
template <typename F>
void parallel_for_threads(int n, const F &fn) {
  if (n <= 1) { fn(0); return; }
  HostPool &pool = HostPool::get();
  auto call = [](const void *o, int k) { (*static_cast<const F *>(o))(k); };
  if (n > pool.workers() + 1 || !pool.run(n, call, &fn))
    for (int k = 0; k < n; k++) fn(k);
}

// Exclusive prefix sum of a[0 .. n) in place, on host threads (per chunk a
// sum, the chunk starts in order, then each chunk's offsets: the result of
// one sequential pass).
inline void scan_exclusive(int *a, long long n) {
  const int nch = layout_threads(n);
  if (nch <= 1) {
    int run = 0;
    for (long long i = 0; i < n; i++) { const int x = a[i]; a[i] = run; run += x; }
    return;
  }
  std::vector<int> part(size_t(nch) + 1, 0);
  parallel_for_threads(nch, [&](int h) {
    const long long c0 = n * h / nch, c1 = n * (h + 1) / nch;
    int s = 0;
    for (long long i = c0; i < c1; i++) s += a[i];
    part[size_t(h) + 1] = s;
  });
  for (int h = 0; h < nch; h++) part[size_t(h) + 1] += part[h];
  parallel_for_threads(nch, [&](int h) {
    const long long c0 = n * h / nch, c1 = n * (h + 1) / nch;
    int run = part[h];
    for (long long i = c0; i < c1; i++) { const int x = a[i]; a[i] = run; run += x; }
  });
}

// o = 0 .. n-1 stably sorted by key(i) in [0, K): a counting sort.  The keys
// (random reads of the constraint records and island tables) on host
// threads; with several threads each counts its range of items per key, the
// (key, thread) counts are scanned in that order and each thread places its
// range -- the order of one sequential pass.  start: scratch.
template <typename Key>
void order_by(int n, int K, const Key &key, std::vector<int> &o, std::vector<int> &k, std::vector<int> &start) {
  k.resize(n);
  o.resize(n);
  const int nth = layout_threads(n);
  parallel_for_threads(nth, [&](int t) {
    const int i0 = int((long long)n * t / nth), i1 = int((long long)n * (t + 1) / nth);
    for (int i = i0; i < i1; i++) k[i] = key(i);
  });
  if (nth <= 1) {
    start.assign(size_t(K) + 1, 0);
    for (int i = 0; i < n; i++) start[size_t(k[i]) + 1]++;
    for (int j = 0; j < K; j++) start[size_t(j) + 1] += start[j];
    for (int i = 0; i < n; i++) o[start[k[i]]++] = i;
    return;
  }
  start.assign(size_t(K) * nth, 0);
  parallel_for_threads(nth, [&](int t) {
    const int i0 = int((long long)n * t / nth), i1 = int((long long)n * (t + 1) / nth);
    int *ct = start.data() + t;
    for (int i = i0; i < i1; i++) ct[size_t(k[i]) * nth]++;
  });
  scan_exclusive(start.data(), (long long)K * nth);
  parallel_for_threads(nth, [&](int t) {
    const int i0 = int((long long)n * t / nth), i1 = int((long long)n * (t + 1) / nth);
    int *ct = start.data() + t;
    for (int i = i0; i < i1; i++) o[ct[size_t(k[i]) * nth]++] = i;
  });
}

// Connected components of nodes 0 .. n-1 under the unions that edges(fn)
// reports (fn(a, b) for every edge; negative ends are ignored), on host
// threads: lock-free union-find whose root is always the smallest node of
// its component (a root is hooked only under a smaller root, with a
// compare-and-swap; finds halve their paths), so the result does not depend
// on the order of the unions.  root[i] = the smallest node of i's component.
// each_edge(t, nth, fn) calls fn for thread t's share of the edges.
template <typename EachEdge>
void components_min_root(int n, int nth, const EachEdge &each_edge, std::vector<int> &root) {
  std::vector<std::atomic<int>> par(static_cast<size_t>(std::max(n, 1)));
  for (int i = 0; i < n; i++) par[size_t(i)].store(i, std::memory_order_relaxed);
  auto find = [&](int x) {
    for (;;) {
      int p = par[size_t(x)].load(std::memory_order_acquire);
      if (p == x) return x;
      const int g = par[size_t(p)].load(std::memory_order_acquire);
      if (g != p) par[size_t(x)].compare_exchange_weak(p, g, std::memory_order_acq_rel);
      x = g;
    }
  };
  auto unite = [&](int a, int b) {
    if (a < 0 || b < 0) return;
    for (;;) {
      a = find(a);
      b = find(b);
      if (a == b) return;
      if (a > b) std::swap(a, b);   // hook the larger root b under the smaller a
      int expect = b;
      if (par[size_t(b)].compare_exchange_strong(expect, a, std::memory_order_acq_rel)) return;
    }
  };
  parallel_for_threads(nth, [&](int t) { each_edge(t, nth, unite); });
  root.resize(size_t(n));
  const int nr = layout_threads(n);
  parallel_for_threads(nr, [&](int t) {
    const int i0 = int((long long)n * t / nr), i1 = int((long long)n * (t + 1) / nr);
    for (int i = i0; i < i1; i++) root[size_t(i)] = find(i);
  });
}

}  // namespace nsn
