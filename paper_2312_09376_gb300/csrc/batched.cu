// Batched RBT solves in one persistent launch (sm_103a).
//
// Thousands of independent systems of uneven order, each with its own seeded
// butterflies, are solved by one kernel: each CTA takes the next system from
// a device work queue (largest first) and runs the whole method on it with
// its threads -- coefficients (Sec. 6), the fused two-sided transform
// (Eq. rbt-depth-d, all layers in one pass), blocked GENP, the transformed
// solve (Eq. precond) and double-precision iterative refinement (Sec. 5) --
// without returning to the host.  The launch is a memset of the queue counter
// plus one kernel (two of each for float with fallback: the double kernel
// then redoes the systems the float kernel, with its double-float fallback,
// left unsolved), so it can be captured in a CUDA graph.  The working
// precision is double or float (then refined to double).
//
// Per-system scratch lives in the caller's workspace at offsets fixed by the
// plan; the descriptor table and the queue order are copied there by
// rbt_solve_batched_plan.  The variant (threads per CTA, GENP block size) is
// chosen by rbt_solve_batched_autotune, which times every compiled variant on
// the planned batch and keeps the fastest for that batch's size histogram.
//
// This file is the host side; the device code is in batched_dev.cuh and the
// kernels are compiled from batched_kernels.cu, one object per working
// precision and variant.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "batched_dev.cuh"

namespace rbt {
namespace bat {

// ------------------------------------------------------------- host side

struct PlanInfo {
    int64_t batch;
    int32_t prec, depth, fallback;
    size_t desc_off, order_off, counter_off, adj_off, sys_off;
    std::string signature;
};

static std::mutex g_mu;
static std::map<const void *, PlanInfo> g_plans;             // by workspace pointer
static std::map<std::string, int> g_tuned;                   // signature -> variant

template <typename T>
static rbt_status launch_variant(int v, const PlanInfo &P, char *w, rbt_batched_info *d_infos, int refine_max,
                                 double tol, cudaStream_t stream, int redo = 0)
{
    BatchedLaunch a;
    a.descs = (const SysDesc *)(w + P.desc_off);
    a.adj = nullptr;
    a.order = (const int *)(w + P.order_off);
    a.batch = (int)P.batch;
    a.counter = (int *)(w + P.counter_off);
    a.infos = d_infos;
    a.sys_base = w + P.sys_off;
    a.depth = P.depth;
    a.refine_max = refine_max;
    a.tol = tol;
    a.fallback = P.fallback;
    a.redo = redo;
    RBT_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int), stream));
    switch (v) {
    case 0: return run_batched<T, 128, 16>(a, stream);
    case 1: return run_batched<T, 128, 32>(a, stream);
    case 2: return run_batched<T, 256, 16>(a, stream);
    default: return run_batched<T, 256, 32>(a, stream);
    }
}

// The whole batch: one launch in double; in float one launch (its fallback
// in double-float inside it) and, with fallback, a second launch of the
// double kernel over the systems still unsolved.
static rbt_status launch_plan(int v, const PlanInfo &P, char *w, rbt_batched_info *d_infos, int refine_max,
                              double tol, cudaStream_t stream)
{
    if (P.prec == RBT_F64) return launch_variant<double>(v, P, w, d_infos, refine_max, tol, stream);
    rbt_status s = launch_variant<float>(v, P, w, d_infos, refine_max, tol, stream);
    if (s != RBT_OK || !P.fallback) return s;
    return launch_variant<double>(v, P, w, d_infos, refine_max, tol, stream, 1);
}

template <typename T> static rbt_status launch_adjoint(int v, const BatchedLaunch &a, cudaStream_t stream)
{
    switch (v) {
    case 0: return run_adjoint<T, 128, 16>(a, stream);
    case 1: return run_adjoint<T, 128, 32>(a, stream);
    case 2: return run_adjoint<T, 256, 16>(a, stream);
    default: return run_adjoint<T, 256, 32>(a, stream);
    }
}

static std::string make_signature(int64_t batch, const int64_t *n, const int64_t *nrhs, int prec, int d)
{
    // histogram of orders in buckets of 64 and of right-hand sides, plus the device
    int hist[64] = {0};
    int64_t maxn = 0, sumr = 0;
    for (int64_t i = 0; i < batch; i++) {
        int b = (int)std::min<int64_t>(n[i] / 64, 63);
        hist[b]++;
        maxn = std::max(maxn, n[i]);
        sumr += nrhs ? nrhs[i] : 1;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    std::string name = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? p.name : "gpu";
    std::string s = name + "|p" + std::to_string(prec) + "|d" + std::to_string(d) + "|b" + std::to_string(batch) +
                    "|r" + std::to_string(sumr) + "|";
    for (int i = 0; i < 64; i++)
        if (hist[i]) s += std::to_string(i) + ":" + std::to_string(hist[i] * 16 / std::max<int64_t>(batch, 1)) + ",";
    return s;
}

}  // namespace bat
}  // namespace rbt

using namespace rbt;
using namespace rbt::bat;

static size_t plan_bytes(const rbt_opts *o, int64_t batch, const int64_t *n, const int64_t *nrhs, size_t *desc_off,
                         size_t *order_off, size_t *counter_off, size_t *adj_off, size_t *sys_off)
{
    size_t off = 0;
    *desc_off = off;
    off = (size_t)align256((int64_t)(off + batch * sizeof(SysDesc)));
    *order_off = off;
    off = (size_t)align256((int64_t)(off + batch * sizeof(int)));
    *counter_off = off;
    off = (size_t)align256((int64_t)(off + 256));
    *adj_off = off;
    off = (size_t)align256((int64_t)(off + batch * sizeof(AdjDesc)));
    *sys_off = off;
    for (int64_t i = 0; i < batch; i++) {
        int64_t r = nrhs ? nrhs[i] : 1;
        // float systems that may fall back keep room for the double-float or double factors
        Layout L = (o->prec == RBT_F64 || o->fallback) ? sys_layout<double>(n[i], r, o->depth)
                                                        : sys_layout<float>(n[i], r, o->depth);
        off += (size_t)L.total;
    }
    return off;
}

extern "C" {

size_t rbt_solve_batched_workspace(const rbt_opts *opts, int64_t batch, const int64_t *n, const int64_t *nrhs)
{
    if (!opts || batch < 0 || (batch > 0 && !n)) return 0;
    size_t a, b, c, d, e;
    return plan_bytes(opts, batch, n, nrhs, &a, &b, &c, &d, &e);
}

rbt_status rbt_solve_batched_plan(const rbt_opts *opts, int64_t batch, const int64_t *n, const int64_t *nrhs,
                                  const double *const *A, const int64_t *lda, const double *const *B,
                                  const int64_t *ldb, double *const *X, const int64_t *ldx, const uint64_t *seeds,
                                  void *work, size_t work_bytes, cudaStream_t stream)
{
    if (!opts || batch < 0 || batch > INT32_MAX) return RBT_ERR_ARG;
    if (opts->prec != RBT_F64 && opts->prec != RBT_F32) return RBT_ERR_UNSUPPORTED;
    if (opts->depth < 0 || opts->depth > 62 || opts->refine_max < 0 || opts->align < 0 || opts->grid_p < 0 ||
        opts->grid_q < 0)
        return RBT_ERR_ARG;
    // batched systems use the non-tiled reference size (no tiles, no process grid)
    if (opts->align > 1 || opts->grid_p > 1 || opts->grid_q > 1) return RBT_ERR_UNSUPPORTED;
    if (opts->kind != RBT_KIND_SCALED && opts->kind != RBT_KIND_ROTATION) return RBT_ERR_ARG;
    if (opts->kind != RBT_KIND_SCALED) return RBT_ERR_UNSUPPORTED;  // batched systems use the scaled butterflies
    if (opts->refine_mode != RBT_REFINE_STATIONARY) return RBT_ERR_UNSUPPORTED;  // stationary steps, then the fallback
    if (batch == 0) return RBT_OK;
    if (!n || !A || !lda || !B || !ldb || !X || !ldx || !work) return RBT_ERR_ARG;
    for (int64_t i = 0; i < batch; i++) {
        int64_t r = nrhs ? nrhs[i] : 1;
        if (n[i] < 1 || r < 1 || lda[i] < n[i] || ldb[i] < n[i] || ldx[i] < n[i] || !A[i] || !B[i] || !X[i])
            return RBT_ERR_ARG;
        if (eff_depth(n[i], opts->depth) > 3 || n[i] > (1 << 20)) return RBT_ERR_UNSUPPORTED;
    }
    PlanInfo P;
    size_t need = plan_bytes(opts, batch, n, nrhs, &P.desc_off, &P.order_off, &P.counter_off, &P.adj_off, &P.sys_off);
    if (work_bytes < need) return RBT_ERR_WORKSPACE;
    P.batch = batch;
    P.prec = opts->prec;
    P.depth = opts->depth;
    P.fallback = opts->fallback ? 1 : 0;
    P.signature = make_signature(batch, n, nrhs, opts->prec, opts->depth);
    std::vector<SysDesc> descs((size_t)batch);
    int64_t off = 0;
    for (int64_t i = 0; i < batch; i++) {
        SysDesc &s = descs[(size_t)i];
        s.n = n[i];
        s.nrhs = nrhs ? nrhs[i] : 1;
        s.A = A[i];
        s.lda = lda[i];
        s.B = B[i];
        s.ldb = ldb[i];
        s.X = X[i];
        s.ldx = ldx[i];
        s.seed = seeds ? seeds[i] : opts->seed + (uint64_t)i;
        s.off = off;
        Layout L = (opts->prec == RBT_F64 || opts->fallback) ? sys_layout<double>(s.n, s.nrhs, opts->depth)
                                                             : sys_layout<float>(s.n, s.nrhs, opts->depth);
        off += L.total;
    }
    // largest systems first: the persistent CTAs then finish together
    std::vector<int> order((size_t)batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    char *w = (char *)work;
    RBT_CUDA_TRY(cudaMemcpyAsync(w + P.desc_off, descs.data(), descs.size() * sizeof(SysDesc), cudaMemcpyHostToDevice,
                                 stream));
    RBT_CUDA_TRY(cudaMemcpyAsync(w + P.order_off, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 stream));
    RBT_CUDA_TRY(cudaStreamSynchronize(stream));  // the host vectors die with this call
    std::lock_guard<std::mutex> lk(g_mu);
    g_plans[work] = P;
    return RBT_OK;
}

rbt_status rbt_solve_batched_run(const rbt_opts *opts, void *work, rbt_batched_info *d_infos, cudaStream_t stream)
{
    if (!opts || !work) return RBT_ERR_ARG;
    PlanInfo P;
    int v = 3;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(work);
        if (it == g_plans.end()) return RBT_ERR_ARG;  // not planned
        P = it->second;
        auto t = g_tuned.find(P.signature);
        if (t != g_tuned.end()) v = t->second;
    }
    if (P.batch == 0) return RBT_OK;
    if (!d_infos) return RBT_ERR_ARG;
    if (opts->prec != P.prec || opts->depth != P.depth || (opts->fallback ? 1 : 0) != P.fallback) return RBT_ERR_ARG;
    return launch_plan(v, P, (char *)work, d_infos, opts->refine_max, opts->tol, stream);
}

rbt_status rbt_solve_batched_autotune(const rbt_opts *opts, void *work, rbt_batched_info *d_infos,
                                      cudaStream_t stream, int32_t *chosen, double *best_ms)
{
    if (!opts || !work || !d_infos) return RBT_ERR_ARG;
    PlanInfo P;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(work);
        if (it == g_plans.end()) return RBT_ERR_ARG;
        P = it->second;
    }
    if (P.batch == 0) return RBT_OK;
    cudaEvent_t e0, e1;
    RBT_CUDA_TRY(cudaEventCreate(&e0));
    RBT_CUDA_TRY(cudaEventCreate(&e1));
    int best = 3;
    float best_t = 1e30f;
    for (int v = 0; v < kNumVariants; v++) {
        for (int rep = 0; rep < 2; rep++) {  // first run warms up
            RBT_CUDA_TRY(cudaEventRecord(e0, stream));
            rbt_status s = launch_plan(v, P, (char *)work, d_infos, opts->refine_max, opts->tol, stream);
            if (s != RBT_OK) return s;
            RBT_CUDA_TRY(cudaEventRecord(e1, stream));
            RBT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            RBT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms < best_t) {
                best_t = ms;
                best = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[P.signature] = best;
    }
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return RBT_OK;
}

rbt_status rbt_solve_batched_adjoint(const rbt_opts *opts, void *work, int64_t batch, const double *const *G,
                                     const int64_t *ldg, double *const *Y, const int64_t *ldy, double *const *GA,
                                     const int64_t *ldga, rbt_batched_info *d_infos, cudaStream_t stream)
{
    if (!opts || !work) return RBT_ERR_ARG;
    PlanInfo P;
    int v = 3;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(work);
        if (it == g_plans.end()) return RBT_ERR_ARG;
        P = it->second;
        auto t = g_tuned.find(P.signature);
        if (t != g_tuned.end()) v = t->second;
    }
    if (batch != P.batch || opts->prec != P.prec || opts->depth != P.depth) return RBT_ERR_ARG;
    if (batch == 0) return RBT_OK;
    if (!G || !ldg || !Y || !ldy || !d_infos || (GA && !ldga)) return RBT_ERR_ARG;
    std::vector<SysDesc> descs((size_t)batch);
    char *w = (char *)work;
    RBT_CUDA_TRY(cudaMemcpyAsync(descs.data(), w + P.desc_off, descs.size() * sizeof(SysDesc), cudaMemcpyDeviceToHost,
                                 stream));
    RBT_CUDA_TRY(cudaStreamSynchronize(stream));
    std::vector<AdjDesc> adj((size_t)batch);
    for (int64_t i = 0; i < batch; i++) {
        const int64_t n = descs[(size_t)i].n;
        if (!G[i] || !Y[i] || ldg[i] < n || ldy[i] < n || (GA && GA[i] && ldga[i] < n)) return RBT_ERR_ARG;
        adj[(size_t)i] = AdjDesc{G[i], ldg[i], Y[i], ldy[i], GA ? GA[i] : nullptr, GA ? ldga[i] : 0};
    }
    RBT_CUDA_TRY(cudaMemcpyAsync(w + P.adj_off, adj.data(), adj.size() * sizeof(AdjDesc), cudaMemcpyHostToDevice,
                                 stream));
    BatchedLaunch a;
    a.descs = (const SysDesc *)(w + P.desc_off);
    a.adj = (const AdjDesc *)(w + P.adj_off);
    a.order = (const int *)(w + P.order_off);
    a.batch = (int)batch;
    a.counter = (int *)(w + P.counter_off);
    a.infos = d_infos;
    a.sys_base = w + P.sys_off;
    a.depth = P.depth;
    a.refine_max = opts->refine_max;
    a.tol = opts->tol;
    a.fallback = P.fallback;
    a.redo = 0;
    RBT_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int), stream));
    rbt_status st = P.prec == RBT_F64 ? launch_adjoint<double>(v, a, stream) : launch_adjoint<float>(v, a, stream);
    if (st != RBT_OK) return st;
    if (P.prec != RBT_F64 && P.fallback) {
        // the systems whose forward solution came from double factors
        a.redo = 1;
        RBT_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int), stream));
        st = launch_adjoint<double>(v, a, stream);
        if (st != RBT_OK) return st;
    }
    RBT_CUDA_TRY(cudaStreamSynchronize(stream));  // the host descriptor vector dies with this call
    return RBT_OK;
}

int32_t rbt_solve_batched_variant(void *work, int32_t *threads, int32_t *nb)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(work);
    if (it == g_plans.end()) return -1;
    int v = 3;
    auto t = g_tuned.find(it->second.signature);
    if (t != g_tuned.end()) v = t->second;
    if (threads) *threads = kVariants[v].nt;
    if (nb) *nb = kVariants[v].nb;
    return v;
}

}  // extern "C"
