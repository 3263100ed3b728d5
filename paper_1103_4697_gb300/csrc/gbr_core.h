// Host-side state of a libgbres context (internal).
#pragma once
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gbres.h"
#include "gbr_internal.h"

namespace gbr {

// A host-side NVTX range for the duration of a scope (a profiler shows it on the
// calling thread's timeline beside the kernels; without one attached each push
// and pop costs a few nanoseconds).  next() closes the current range and opens
// the following phase's, so early returns always leave the ranges balanced.
class NvtxScope {
  public:
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    void next(const char *name) {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

// First-fit allocator with coalescing over one device allocation (the caller's
// workspace or the library's own cudaMalloc of the budget).  256-byte aligned.
class Arena {
   public:
    void init(void *base, size_t cap);
    void *alloc(size_t bytes);   // nullptr when no free block is large enough
    void release(void *p);
    size_t largest_free();
    size_t in_use() {
        std::lock_guard<std::mutex> g(mu);
        return inuse;
    }
    size_t peak_use() {
        std::lock_guard<std::mutex> g(mu);
        return peak;
    }
    size_t capacity() const { return cap; }

   private:
    char *base = nullptr;
    size_t cap = 0, inuse = 0, peak = 0;
    std::map<size_t, size_t> free_, used_;
    std::mutex mu;
};

struct ServeState;   // gbr_serve.cu

}  // namespace gbr

struct gbr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    void *ws = nullptr;
    bool own_ws = false;
    size_t budget = 0;
    gbr::Arena arena;
    std::mutex mu;                 // serialises synchronous calls
    std::mutex err_mu;
    std::string err;
    ModP *d_mods = nullptr;
    double *d_l2pref = nullptr;         // sum_{i<k} log2 p_i, k = 0..num_primes (the step graphs' plan check)
    int32_t *d_err = nullptr;
    uint32_t *d_garner = nullptr;
    int garner_K = 0;
    uint32_t *d_crtw = nullptr;          // warp Chinese remaindering tables (crt_warp_table)
    int crtw_K = 0;
    uint32_t *d_invk = nullptr;
    int invk_K = 0, invk_T = 0;
    void *h_pin[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t h_pin_cap[4] = {0, 0, 0, 0};
    cudaEvent_t ev[8] = {};
    int drop_unlucky = 0, stats_on = 0, graph_on = 1, extra_primes = 0, gemm_on = 1, reg_on = 1, tc_on = 1;
    int pts_mode = 0;   // GBR_OPT_POINTS: 0 chosen per pair by cost, 1 integer points, 2 roots of unity
    gbr_stats stats{};
    std::map<uint64_t, cudaGraphExec_t> graphs;
    struct Vinv {
        uint32_t *d = nullptr;
        uint16_t *tc = nullptr;   // bf16 digit tiles for the tensor-core path (built on first use)
        int K = 0;
        size_t bytes = 0;
        uint64_t last_use = 0;
    };
    std::map<int64_t, Vinv> vinv;  // inverse Vandermonde matrices, key 4 n + point-set mode
    std::vector<gbr_resident *> shots;   // idle one-shot batches, oldest first (a repeated shape class reuses one)
    uint64_t vinv_clock = 0, vinv_run_mark = 0;
    const uint32_t *get_vinv(int n, int K, int mode);   // nullptr if it cannot be built
    const uint16_t *get_vinv_tc(int n, int K, int mode);   // digit tiles of a matrix get_vinv returned
    gbr::ServeState *serve = nullptr;
    gbr_ctx *pipe[2] = {nullptr, nullptr};   // private workers that pipeline large one-shot batches
    gbr_ctx *mixw = nullptr;                 // private worker for the gcd half of gbr_mixed_batch
    int64_t gcd_kernels = 0, gcd_subproblems = 0, gcd_h2d = 0, gcd_d2h = 0;   // counters of the last gcd call
    int pipe_on = 1;
    std::map<int, int> tuned_evalres;   // degree bucket -> block size chosen by the autotuner
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    cudaError_t capture_stream_ready();
    void autotune_load();
    void autotune_record(const char *kernel, int key, int value);
    gbr_ctx *parent = nullptr;     // serving workers share the parent's arena
    bool own_stream = false;

    int fail(int code, const char *what, cudaError_t e = cudaSuccess);
    void *dalloc(size_t bytes);
    void dfree(void *p);
    gbr::Arena &mem() { return parent ? parent->arena : arena; }
    void *pinned(size_t bytes, int slot);   // grow-only pinned staging buffer per slot
    int ensure_tables(int K, int T, int KW = 0);   // KW: primes of the warp Chinese remaindering
};

struct gbr_resident {
    int n = 0, var = 1, disc = 0;
    int64_t coef_words = 0, rowdeg_n = 0, upload_bytes = 0;
    uint64_t *d_coef = nullptr;
    gbr::PairDesc *d_desc = nullptr;
    int32_t *d_rowdeg = nullptr;
    gbr::PairBound *d_bounds = nullptr;
    int32_t *d_deg = nullptr;
    std::vector<gbr::PairDesc> h_desc;
    std::vector<gbr::PairPlan> h_plan;
    std::vector<double> h_log2B;        // the device's coefficient bound per job (log2)
    std::vector<int32_t> h_deg;         // the degree bound per job (the plan's points may be more)
    std::vector<char> h_blk;            // host copy of the last plan block (storage reused)
    char *d_planblk = nullptr;
    size_t planblk_cap = 0;
    uint32_t *d_res = nullptr, *d_val = nullptr, *d_cf = nullptr, *d_out = nullptr, *d_den = nullptr;
    size_t res_cap = 0, val_cap = 0, cf_cap = 0, out_cap = 0, den_cap = 0;
    int8_t *d_sign = nullptr;
    size_t sign_cap = 0;
    uint8_t *d_flags = nullptr;
    size_t flags_cap = 0;
    uint32_t *d_gtab = nullptr;
    size_t gtab_cap = 0;
    char *d_redo = nullptr;   // register-form redo counters and warp lists
    size_t redo_cap = 0;
    int64_t out_words = 0, sign_bytes = 0;
    bool ran = false;
    bool oneshot = false;               // created by a one-shot call: never captured
    const void *shot_src = nullptr;     // one-shot cache: the host input of the call that last used it
    cudaGraphExec_t gexec = nullptr;    // captured device stages of the last plan
    int gstate = 0;                     // 0 no plan, 1 plan run once, 2 captured
    int64_t graph_kernels = 0;
    std::vector<uintptr_t> gkey;        // pointers and launch shapes of the captured plan
    std::vector<char> gblk;             // plan block of the captured plan
    // the whole step as one graph (bounds, plan check, stages), captured once the
    // stage graph has replayed: later runs launch it with no host planning in
    // between; the stages return at once if the fresh bounds no longer fit the plan
    cudaGraphExec_t fexec = nullptr;
    int fstate = 0;                     // 0 none, 2 captured and valid for fsig
    std::vector<uintptr_t> fsig;        // options and table pointers the step graph assumes
    std::vector<std::pair<int64_t, std::pair<const void *, const void *>>> fvinv;   // cached matrices it reads
    gbr_stats fast_st{};
    int fast_nredo = 0;
    int64_t fast_out_w = 0, fast_sign_b = 0, fast_kernels = 0;
    bool fast_pending = false;          // the pending run is a step-graph launch
    // launched but not yet finished (gbr_run_resident_launch / _finish)
    bool pending = false;
    gbr_stats pend_st{};
    int pend_nredo = 0;
    int64_t pend_out_w = 0, pend_sign_b = 0;
};

// internal entry points (context lock held by the caller)
int gbr_run_resident_locked(gbr_ctx *c, gbr_resident *r);
int gbr_run_resident_launch(gbr_ctx *c, gbr_resident *r);   // bounds, plan, stages enqueued
int gbr_run_resident_finish(gbr_ctx *c, gbr_resident *r);   // wait, check, statistics
int gbr_fetch_resident_locked(gbr_ctx *c, gbr_resident *r, int first, int count, gbr_bigpoly *out);
void gbr_free_resident_locked(gbr_ctx *c, gbr_resident *r);
void gbr_free_shots(gbr_ctx *c);   // the context's idle one-shot batches
void gbr_serve_shutdown(gbr_ctx *c);
void gbr_parallel_for(int n, int threads, const std::function<void(int, int)> &fn);   // fn(lo, hi) on threads
bool gbr_alloc_results(gbr_bigpoly *out, int count);
// gcd batch with optional cofactors (out_a = p / gcd, out_b = q / gcd; both or
// neither), with the context lock held
int gbr_gcd_cof_locked(gbr_ctx *c, int n, const gbr_upoly *p, const gbr_upoly *q, gbr_bigpoly *out,
                       gbr_bigpoly *out_a, gbr_bigpoly *out_b);   // one refcounted host block for a call's results
char *gbr_pinned_result_block(size_t bytes, size_t *got);
void gbr_register_result_block(char *base, size_t size, int64_t refs, bool pinned);
gbr_ctx *gbr_make_worker(gbr_ctx *parent);    // own stream and tables, parent's arena
// gbr_resultant_info, with the summed forms of the bound (small shapes) or without them
int resultant_info_impl(const gbr_bipoly *f, const gbr_bipoly *g, int var, int disc, gbr_res_info *out, bool summed);
void gbr_destroy_worker(gbr_ctx *w);
