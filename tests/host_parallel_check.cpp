// Checks the host-side parallel passes of the layout build (nsn_hostpar.h)
// against their sequential definitions: the stable counting sort against
// std::stable_sort, the exclusive scan against a running sum, the parallel
// union-find against a sequential one, every item of a pass run exactly
// once, from two calling threads at once, from inside a pass and in a child
// forked after the workers started.  Prints "ok" and exits 0, else names the first failure.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <random>
#include <vector>

#include <sys/wait.h>
#include <unistd.h>

#include "nsn_hostpar.h"

using namespace nsn;

int main() {
  std::mt19937 rng(7);
  for (int trial = 0; trial < 30; trial++) {
    const int n = trial % 6 == 0 ? int(rng() % 5000) : 100000 + int(rng() % 700000);
    const int K = 1 + int(rng() % (trial % 2 ? 64 : 200000));
    std::vector<int> keys(n), o, k, scratch, ref(n);
    for (int &x : keys) x = int(rng() % K);
    order_by(n, K, [&](int i) { return keys[i]; }, o, k, scratch);
    for (int i = 0; i < n; i++) ref[i] = i;
    std::stable_sort(ref.begin(), ref.end(), [&](int a, int b) { return keys[a] < keys[b]; });
    if (o != ref) { std::printf("order_by differs: n %d K %d\n", n, K); return 1; }
  }
  for (long long n : {0LL, 1LL, 1000LL, 3000001LL}) {
    std::vector<int> a(static_cast<size_t>(n)), b;
    for (int &x : a) x = int(rng() % 9);
    b = a;
    int run = 0;
    for (int &x : b) { const int y = x; x = run; run += y; }
    scan_exclusive(a.data(), n);
    if (a != b) { std::printf("scan differs: n %lld\n", n); return 1; }
  }
  for (int n = 1; n <= 40; n++) {
    std::vector<int> hit(static_cast<size_t>(n), 0);
    parallel_for_threads(n, [&](int q) { hit[size_t(q)]++; });
    for (int q = 0; q < n; q++)
      if (hit[size_t(q)] != 1) { std::printf("item %d of %d ran %d times\n", q, n, hit[size_t(q)]); return 1; }
  }
  // components: against a sequential union-find (root = smallest node)
  for (int trial = 0; trial < 12; trial++) {
    const int n = 1000 + int(rng() % 200000), m = int(rng() % (2 * n));
    std::vector<std::pair<int, int>> edges(static_cast<size_t>(m));
    for (auto &e : edges) {
      e.first = int(rng() % n) - (rng() % 50 == 0 ? n : 0);   // some ends negative (ignored)
      e.second = trial % 2 ? int(rng() % n) : std::min(n - 1, std::max(0, e.first + int(rng() % 9) - 4));
    }
    std::vector<int> ref(static_cast<size_t>(n));
    for (int i = 0; i < n; i++) ref[size_t(i)] = i;
    auto f = [&](int x) { while (ref[size_t(x)] != x) x = ref[size_t(x)] = ref[size_t(ref[size_t(x)])]; return x; };
    for (auto &e : edges) {
      if (e.first < 0 || e.second < 0) continue;
      int a = f(e.first), b = f(e.second);
      if (a == b) continue;
      if (a < b) ref[size_t(b)] = a; else ref[size_t(a)] = b;
    }
    for (int i = 0; i < n; i++) ref[size_t(i)] = f(i);
    std::vector<int> root;
    components_min_root(n, layout_threads(m), [&](int t, int nth, auto &&unite) {
      const long long e0 = (long long)m * t / nth, e1 = (long long)m * (t + 1) / nth;
      for (long long e = e0; e < e1; e++) unite(edges[size_t(e)].first, edges[size_t(e)].second);
    }, root);
    if (root != ref) { std::printf("components differ: n %d m %d\n", n, m); return 1; }
  }
  std::atomic<int> bad{0};
  auto user = [&] {
    for (int pass = 0; pass < 2000; pass++) {
      std::vector<int> hit(12, 0);
      parallel_for_threads(12, [&](int q) { hit[size_t(q)]++; });
      for (int x : hit) bad += x != 1;
    }
  };
  std::thread t1(user), t2(user);
  t1.join();
  t2.join();
  std::vector<int> outer(8, 0);
  parallel_for_threads(8, [&](int q) {
    std::vector<int> in(4, 0);
    parallel_for_threads(4, [&](int r) { in[size_t(r)] = 1; });
    outer[size_t(q)] = in[0] + in[1] + in[2] + in[3];
  });
  for (int x : outer) bad += x != 4;
  // a child forked after the workers started runs its passes on its own thread
  {
    const pid_t child = fork();
    if (child == 0) {
      std::vector<int> hit(12, 0);
      parallel_for_threads(12, [&](int q) { hit[size_t(q)]++; });
      int ok = 1;
      for (int x : hit) ok &= x == 1;
      _exit(ok ? 0 : 1);
    }
    int status = 0;
    waitpid(child, &status, 0);
    if (!WIFEXITED(status) || WEXITSTATUS(status) != 0) { std::printf("forked child failed\n"); return 1; }
  }
  if (bad) { std::printf("%d items ran other than once\n", bad.load()); return 1; }
  std::printf("ok\n");
  return 0;
}
