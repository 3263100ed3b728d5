// Test harness (CPU): the host worker pool behind gbr_parallel_for, driven from
// several threads at once with nested calls; every index must be visited exactly
// once.  Built against libgbres.so and run by test_host_native.py; prints "bad N".
#include <atomic>
#include <cstdio>
#include <functional>
#include <thread>
#include <vector>

void gbr_parallel_for(int n, int threads, const std::function<void(int, int)> &fn);

int main() {
    std::atomic<long> bad{0};
    std::vector<std::thread> callers;
    for (int c = 0; c < 4; ++c)
        callers.emplace_back([&, c] {
            for (int it = 0; it < 1500; ++it) {
                const int n = (it * 37 + c) % 5000;
                std::vector<int> hit(n, 0);
                gbr_parallel_for(n, 16, [&](int lo, int hi) {
                    for (int i = lo; i < hi; ++i) hit[i]++;
                    if (it % 100 == 0) gbr_parallel_for(10, 4, [](int, int) {});   // nested: runs inline
                });
                for (int i = 0; i < n; ++i)
                    if (hit[i] != 1) bad++;
            }
        });
    for (auto &t : callers) t.join();
    std::printf("bad %ld\n", bad.load());
    return 0;
}
