// Host drivers: GENP dispatch by precision and the whole RBT solve with
// iterative refinement and the double-precision fallback.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "genp_internal.cuh"
#include "gemm_tc.cuh"
#include "df64.cuh"

namespace rbt {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- bounded waits: limit and test stall (rbt_debug_*)
static std::atomic<long long> g_wait_ns{kDefaultWaitNs};
static std::atomic<int> g_stall{RBT_STALL_NONE};
long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }
int debug_stall() { return g_stall.load(std::memory_order_relaxed); }

// ---- instrumentation: event pairs per class, resolved on read
struct ProfEvent {
    int cls;
    cudaEvent_t e0, e1;
};
static std::mutex g_prof_mu;
static std::vector<ProfEvent> g_prof;
static std::vector<cudaEvent_t> g_prof_pool;
static ProfEvent g_prof_open[kProfClasses];
static bool g_prof_has_open[kProfClasses];
static std::atomic<bool> g_prof_enabled{false};
static double g_prof_ms[kProfClasses];
static long long g_prof_n[kProfClasses];

bool prof_on() { return g_prof_enabled.load(std::memory_order_relaxed); }

static cudaEvent_t prof_event()
{
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void prof_resolve_locked()
{
    for (auto &p : g_prof) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            g_prof_ms[p.cls] += ms;
            g_prof_n[p.cls] += 1;
        }
        g_prof_pool.push_back(p.e0);
        g_prof_pool.push_back(p.e1);
    }
    g_prof.clear();
}

void prof_record(int cls, cudaStream_t s, bool begin)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (begin) {
        ProfEvent p{cls, prof_event(), prof_event()};
        cudaEventRecord(p.e0, s);
        g_prof_open[cls] = p;
        g_prof_has_open[cls] = true;
    } else if (g_prof_has_open[cls]) {
        ProfEvent p = g_prof_open[cls];
        g_prof_has_open[cls] = false;
        cudaEventRecord(p.e1, s);
        g_prof.push_back(p);
        if (g_prof.size() > 4096) prof_resolve_locked();
    }
}

static int default_nb(int prec)
{
    return (prec == RBT_F64 || is_df64_storage(prec)) ? kDefaultNB64 : kDefaultNB32;
}

size_t genp_factor_workspace_impl(int64_t n, int prec, int nb)
{
    if (n <= 0) return 0;
    if (nb == 0) nb = default_nb(prec);
    if (prec == RBT_TF32 || prec == RBT_BF16) return tc_update_workspace(n, prec, nb);
    if (is_sliced(prec)) return oz_factor_workspace(n);
    return 0;
}

rbt_status genp_factor_impl(int64_t n, int prec, void *A, int64_t lda, int64_t *info, void *work,
                            size_t work_bytes, int nb, cudaStream_t stream)
{
    if (nb == 0) nb = default_nb(prec);
    rbt_status st = genp_configure(prec, nb);
    if (st != RBT_OK) return st;
    if (prec == RBT_F64) return genp_panel_steps<double>(n, (double *)A, lda, info, nb, 0, n, true, stream);
    if (prec == RBT_DF64) return genp_panel_steps<df64>(n, (df64 *)A, lda, info, nb, 0, n, true, stream);
    if (is_sliced(prec))
        return genp_factor_oz(n, (df64 *)A, lda, info, work, work_bytes, sliced_digits(prec), stream);
    if (prec == RBT_F32) return genp_panel_steps<float>(n, (float *)A, lda, info, nb, 0, n, true, stream);
    return genp_factor_tc(n, prec, (float *)A, lda, info, work, work_bytes, nb, stream);
}

}  // namespace rbt

using namespace rbt;

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid_opts(const rbt_opts *o)
{
    return o && o->depth >= 0 && o->depth <= 62 && o->prec >= RBT_F64 && o->prec <= kLastPrec &&
           o->refine_max >= 0 && o->nb >= 0 && o->nb <= kMaxNB && !(o->tol < 0) && o->align >= 0 &&
           (o->refine_mode == RBT_REFINE_STATIONARY || o->refine_mode == RBT_REFINE_GMRES) && o->restart >= 0 &&
           o->restart <= kGmresMaxRestart && (o->kind == RBT_KIND_SCALED || o->kind == RBT_KIND_ROTATION) &&
           o->grid_p >= 0 && o->grid_q >= 0 && o->grid_p <= kMaxGridSide && o->grid_q <= kMaxGridSide &&
           rbt_reference_size(0, o->depth, o->align, o->grid_p, o->grid_q) >= 0;
}

}  // namespace

namespace rbt {

void solve_layout(const rbt_opts *o, int64_t n, int64_t nrhs, SolveLayout *out)
{
    SolveLayout &L = *out;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    L.ldt = (int64_t)align_up((size_t)(n > 0 ? n : 1), 32);
    size_t es = (o->prec == RBT_F64 || is_df64_storage(o->prec)) ? 8 : 4;
    size_t nn = (size_t)L.ldt * (size_t)(n > 0 ? n : 1);
    int64_t d = o->depth > 0 ? o->depth : 1;
    int64_t nr = nrhs > 0 ? nrhs : 1;
    L.at = take(nn * es);
    L.at64 = (o->fallback && o->prec != RBT_F64) ? take(nn * 8) : (size_t)-1;
    L.u = take((size_t)n * d * 8);
    L.v = take((size_t)n * d * 8);
    L.r = take((size_t)n * nr * 8);
    L.info = take(8);
    L.scal = take(4 * 8);
    L.res = take(residual_ws(n, nr));
    L.fac = take(genp_factor_workspace_impl(n, o->prec, o->nb));
    size_t sol_ws = genp_solve_workspace(n, nr, o->prec) + genp_solve_workspace(n, nr, RBT_F32);
    if (o->refine_mode == RBT_REFINE_GMRES) sol_ws = std::max(sol_ws, genp_solve_wp_workspace(n, 1));
    L.sol = take(sol_ws);
    if (o->refine_mode == RBT_REFINE_GMRES) {
        // basis Q (m + 1 columns), z, w, a zero vector, dot-product partials, h / y
        const int64_t m = o->restart > 0 ? o->restart : kGmresDefaultRestart;
        const size_t nv = (size_t)(n > 0 ? n : 1);
        L.gm = take(8 * (nv * (size_t)(m + 4) + (size_t)(m + 1) * (size_t)gm_part_len(n) + 4 * (size_t)(m + 2)));
    } else {
        L.gm = (size_t)-1;
    }
    L.total = off;
}

}  // namespace rbt

namespace {

SolveLayout plan(const rbt_opts *o, int64_t n, int64_t nrhs)
{
    SolveLayout L;
    solve_layout(o, n, nrhs, &L);
    return L;
}

rbt_status read_pivot_status(int64_t k, int prec, const void *At, int64_t ldt, cudaStream_t s, rbt_status *out)
{
    double p = 0.0;
    if (prec == RBT_F64) {
        RBT_CUDA_TRY(cudaMemcpyAsync(&p, (const double *)At + k + k * ldt, 8, cudaMemcpyDeviceToHost, s));
    } else if (is_df64_storage(prec)) {
        float f[2] = {0.f, 0.f};
        RBT_CUDA_TRY(cudaMemcpyAsync(f, (const float *)At + 2 * (k + k * ldt), 8, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaStreamSynchronize(s));
        p = (double)f[0] + (double)f[1];
        if (!std::isfinite(f[0]) || !std::isfinite(f[1])) p = NAN;
    } else {
        float f = 0.f;
        RBT_CUDA_TRY(cudaMemcpyAsync(&f, (const float *)At + k + k * ldt, 4, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaStreamSynchronize(s));
        p = f;
    }
    RBT_CUDA_TRY(cudaStreamSynchronize(s));
    *out = (p == 0.0) ? RBT_ZERO_PIVOT : RBT_NONFINITE;
    return RBT_OK;
}

// dX = V A~^{-1} U^T R, in place in R
rbt_status correction(int64_t n, int64_t nrhs, int d, int64_t align, int kind, const double *U, const double *V, int prec,
                      const void *At, int64_t ldt, double *R, int64_t ldr, void *sol, size_t sol_bytes,
                      cudaStream_t s)
{
    rbt_status st = apply_vec(n, d, align, U, n, 1, R, ldr, nrhs, s, kind);
    if (st != RBT_OK) return st;
    (void)sol_bytes;  // sized by the solve layout
    st = genp_solve_run(n, nrhs, prec, At, ldt, 0, R, ldr, sol, s);
    if (st != RBT_OK) return st;
    return apply_vec(n, d, align, V, n, 0, R, ldr, nrhs, s, kind);
}

// z <- V A~^{-1} U^T z for one column in double arithmetic with the stored
// factors: the preconditioner M^{-1} of GMRES-based refinement, applied in
// the working precision so that it is the same linear operator every time.
rbt_status precondition_wp(int64_t n, int d, int64_t align, int kind, const double *U, const double *V, int prec,
                           const void *At, int64_t ldt, double *z, void *sol, size_t sol_bytes, cudaStream_t s)
{
    rbt_status st = apply_vec(n, d, align, U, n, 1, z, n, 1, s, kind);
    if (st != RBT_OK) return st;
    (void)sol_bytes;  // sized by the solve layout
    st = genp_solve_wp_run(n, 1, prec, At, ldt, 0, z, n, sol, s);
    if (st != RBT_OK) return st;
    return apply_vec(n, d, align, V, n, 0, z, n, 1, s, kind);
}

// One GMRES cycle for column x (residual r = b - A x given): restarted GMRES
// of at most m steps on A M^{-1} u = r with M^{-1} = V A~^{-1} U^T, the
// Arnoldi vectors orthogonalized by classical Gram-Schmidt applied twice,
// then x += M^{-1} Q y.  Adds the preconditioned products used to *used.
rbt_status gmres_cycle(int64_t n, int d, int64_t align, int kind, const double *U, const double *V, int prec, const void *At,
                       int64_t ldt, void *sol, size_t sol_bytes, const double *A, int64_t lda,
                       const double *d_anorm, double *res_part, const double *r, double *x, int m, char *gw,
                       cudaStream_t s, int *used)
{
    const int64_t nblk = gm_part_len(n);
    double *Q = (double *)gw;
    double *z = Q + (size_t)n * (m + 1);
    double *w = z + n;
    double *zero = w + n;
    double *part = zero + n;
    double *dh = part + (size_t)(m + 1) * nblk;  // [0, m+1) first pass, [m+2, 2m+3) second pass
    double *dscr = dh + 2 * (m + 2);              // residual-kernel scratch (its backward error)
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0), y(m), h1(m + 2), h2(m + 2);
    auto HH = [&](int i, int j) -> double & { return H[(size_t)i + (size_t)j * (m + 1)]; };
    int wait_flag = 0;  // the chained triangular solves' timeout flag (front of their scratch)
    rbt_status st;
    RBT_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(double) * n, s));
    st = gm_dots(n, r, n, 1, r, part, dh, s);
    if (st != RBT_OK) return st;
    double beta2 = 0.0;
    RBT_CUDA_TRY(cudaMemcpyAsync(&beta2, dh, 8, cudaMemcpyDeviceToHost, s));
    RBT_CUDA_TRY(cudaStreamSynchronize(s));
    const double beta = std::sqrt(beta2);
    if (!(beta > 0.0) || !std::isfinite(beta)) return RBT_OK;
    st = gm_scale(n, 1.0 / beta, r, Q, s);
    if (st != RBT_OK) return st;
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; j++) {
        // w = A M^{-1} q_j
        RBT_CUDA_TRY(cudaMemcpyAsync(z, Q + (size_t)j * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        st = precondition_wp(n, d, align, kind, U, V, prec, At, ldt, z, sol, sol_bytes, s);
        if (st != RBT_OK) return st;
        st = residual_impl(n, 1, A, lda, z, n, zero, n, w, n, d_anorm, dscr, res_part, s);  // w = -A z
        if (st != RBT_OK) return st;
        st = gm_scale(n, -1.0, w, w, s);
        if (st != RBT_OK) return st;
        ++*used;
        // classical Gram-Schmidt, twice
        st = gm_dots(n, Q, n, j + 1, w, part, dh, s);
        if (st == RBT_OK) st = gm_sub(n, Q, n, j + 1, dh, w, s);
        if (st == RBT_OK) st = gm_dots(n, Q, n, j + 1, w, part, dh + (m + 2), s);
        if (st == RBT_OK) st = gm_sub(n, Q, n, j + 1, dh + (m + 2), w, s);
        if (st == RBT_OK) st = gm_dots(n, w, n, 1, w, part, dh + (m + 1), s);
        if (st != RBT_OK) return st;
        RBT_CUDA_TRY(cudaMemcpyAsync(h1.data(), dh, sizeof(double) * (m + 2), cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaMemcpyAsync(h2.data(), dh + (m + 2), sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaMemcpyAsync(&wait_flag, sol, 4, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaStreamSynchronize(s));
        if (wait_flag) return RBT_ERR_TIMEOUT;
        for (int i = 0; i <= j; i++) HH(i, j) = h1[i] + h2[i];
        const double hn = std::sqrt(h1[m + 1]);
        HH(j + 1, j) = hn;
        if (hn > 0.0 && std::isfinite(hn)) {
            st = gm_scale(n, 1.0 / hn, w, Q + (size_t)(j + 1) * n, s);
            if (st != RBT_OK) return st;
        }
        for (int i = 0; i < j; i++) {  // earlier rotations on the new column
            const double a = HH(i, j), b = HH(i + 1, j);
            HH(i, j) = cs[i] * a + sn[i] * b;
            HH(i + 1, j) = -sn[i] * a + cs[i] * b;
        }
        const double a = HH(j, j), b = HH(j + 1, j);
        const double rr = std::sqrt(a * a + b * b);
        if (!(rr > 0.0) || !std::isfinite(rr)) break;  // a zero (or non-finite) column: keep the first j steps
        cs[j] = a / rr;
        sn[j] = b / rr;
        HH(j, j) = rr;
        HH(j + 1, j) = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k = j + 1;
        if (!(hn > 0.0) || !std::isfinite(hn) || std::fabs(g[j + 1]) <= 1e-14 * beta) break;
    }
    // y = R^{-1} g, x += M^{-1} (Q y)
    for (int i = k - 1; i >= 0; i--) {
        double t = g[i];
        for (int c = i + 1; c < k; c++) t -= HH(i, c) * y[c];
        y[i] = t / HH(i, i);
    }
    RBT_CUDA_TRY(cudaMemcpyAsync(dh, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    st = gm_gemv(n, Q, n, k, dh, z, s);
    if (st != RBT_OK) return st;
    st = precondition_wp(n, d, align, kind, U, V, prec, At, ldt, z, sol, sol_bytes, s);
    if (st != RBT_OK) return st;
    st = gm_add(n, z, x, s);
    if (st != RBT_OK) return st;
    RBT_CUDA_TRY(cudaStreamSynchronize(s));  // y lives on this host stack until the copy is done
    return RBT_OK;
}

}  // namespace

extern "C" {

uint64_t rbt_kernel_launches(void) { return (uint64_t)g_launches.load(); }

int64_t rbt_debug_wait_limit(int64_t ns)
{
    return (int64_t)g_wait_ns.exchange(ns > 0 ? (long long)ns : kDefaultWaitNs);
}

int32_t rbt_debug_stall(int32_t which)
{
    const int v = (which == RBT_STALL_CHAIN || which == RBT_STALL_OZ_COPY) ? which : RBT_STALL_NONE;
    return (int32_t)g_stall.exchange(v);
}

void rbt_prof_enable(int32_t on) { g_prof_enabled.store(on != 0); }

void rbt_prof_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_resolve_locked();
    for (int c = 0; c < kProfClasses; c++) {
        g_prof_ms[c] = 0.0;
        g_prof_n[c] = 0;
    }
}

rbt_status rbt_prof_read(int32_t cls, double *ms, int64_t *launches)
{
    if (cls < 0 || cls >= kProfClasses || !ms || !launches) return RBT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_resolve_locked();
    *ms = g_prof_ms[cls];
    *launches = g_prof_n[cls];
    return RBT_OK;
}

size_t rbt_solve_workspace(const rbt_opts *opts, int64_t n, int64_t nrhs)
{
    if (!valid_opts(opts) || n < 0 || nrhs < 0) return 0;
    return plan(opts, n, nrhs).total;
}

rbt_status rbt_solve(const rbt_opts *opts, int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double *X, int64_t ldx, void *work, size_t work_bytes, rbt_info *info,
                     cudaStream_t s)
{
    if (info) {
        info->status = RBT_ERR_ARG;
        info->zero_pivot = -1;
        info->iters = 0;
        info->fell_back = 0;
        info->berr_unrefined = NAN;
        info->berr = NAN;
    }
    int64_t mn = n > 1 ? n : 1;
    if (!valid_opts(opts) || !info || n < 0 || nrhs < 0 || lda < mn || ldb < mn || ldx < mn) return RBT_ERR_ARG;
    if (n == 0 || nrhs == 0) {
        info->status = RBT_OK;
        info->berr = info->berr_unrefined = 0.0;
        return RBT_OK;
    }
    if (!A || !B || !X || !work) return RBT_ERR_ARG;
    const int prec = opts->prec, d = opts->depth;
    if (prec != RBT_F64 && eff_depth(n, d) > 3) return RBT_ERR_UNSUPPORTED;
    if (rbt_reference_size(n, d, opts->align, opts->grid_p, opts->grid_q) < 0) return RBT_ERR_ARG;
    // tile size and process grid fold into one alignment of the reference size
    const int64_t align = effective_align(opts->align, opts->grid_p, opts->grid_q);
    SolveLayout L = plan(opts, n, nrhs);
    if (work_bytes < L.total) return RBT_ERR_WORKSPACE;
    char *w = (char *)work;
    void *At = w + L.at;
    double *At64 = L.at64 != (size_t)-1 ? (double *)(w + L.at64) : nullptr;
    double *U = (double *)(w + L.u), *V = (double *)(w + L.v), *R = (double *)(w + L.r);
    int64_t *d_info = (int64_t *)(w + L.info);
    double *scal = (double *)(w + L.scal);  // [0] ||A||, [1] berr
    double *res = (double *)(w + L.res);
    void *fac = w + L.fac;
    void *sol = w + L.sol;
    size_t fac_bytes = L.sol - L.fac, sol_bytes = L.total - L.sol;
    const int64_t ldt = L.ldt;
    rbt_status st;

    // the chained solves' timeout flag (front of their scratch) is cleared once
    // here and read after every step: a timeout anywhere in this call sticks
    RBT_CUDA_TRY(cudaMemsetAsync(sol, 0, sizeof(int), s));

    // 1. butterflies and the transformed working matrix (Eq. precond step 1)
    st = opts->kind == RBT_KIND_ROTATION ? rbt_generate_rot(n, d, align, opts->seed, U, V, n, s)
                                         : rbt_generate(n, d, opts->seed, U, V, n, s);
    if (st != RBT_OK) return st;
    st = apply_2sided_wp(n, d, align, U, V, n, A, lda, At, ldt, prec, s, opts->kind);
    if (st != RBT_OK) return st;
    st = norm_inf_impl(n, A, lda, scal, res, s);
    if (st != RBT_OK) return st;

    // 2. GENP of A~ (step 2)
    st = genp_factor(n, prec, At, ldt, d_info, fac, fac_bytes, opts->nb, s);
    if (st != RBT_OK) return st;

    // 3. x = V A~^{-1} U^T b (steps 1-3), residual and backward error
    RBT_CUDA_TRY(cudaMemcpy2DAsync(X, ldx * 8, B, ldb * 8, n * 8, nrhs, cudaMemcpyDeviceToDevice, s));
    st = correction(n, nrhs, d, align, opts->kind, U, V, prec, At, ldt, X, ldx, sol, sol_bytes, s);
    if (st != RBT_OK) return st;
    st = residual_impl(n, nrhs, A, lda, X, ldx, B, ldb, R, n, scal, scal + 1, res, s);
    if (st != RBT_OK) return st;
    int64_t h_info = -1;
    double berr = 0.0;
    int h_wait = 0;  // the chained triangular solves' timeout flag (front of their scratch)
    RBT_CUDA_TRY(cudaMemcpyAsync(&h_info, d_info, 8, cudaMemcpyDeviceToHost, s));
    RBT_CUDA_TRY(cudaMemcpyAsync(&berr, scal + 1, 8, cudaMemcpyDeviceToHost, s));
    RBT_CUDA_TRY(cudaMemcpyAsync(&h_wait, sol, 4, cudaMemcpyDeviceToHost, s));
    RBT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_wait) return RBT_ERR_TIMEOUT;
    if (h_info == -2) return RBT_ERR_TIMEOUT;

    int cur_prec = prec;
    const void *cur_At = At;
    int64_t cur_ldt = ldt;
    int fell_back = 0;  // rbt_info.fell_back: 1 = double refactorization, 2 = eight-digit one
    if (h_info >= 0) {
        rbt_status ps;
        st = read_pivot_status(h_info, prec, At, ldt, s, &ps);
        if (st != RBT_OK) return st;
        if (prec == RBT_F64 || !opts->fallback || !At64) {
            info->status = ps;
            info->zero_pivot = h_info;
            return ps;
        }
        berr = INFINITY;  // a failed low-precision factor counts as a stall
    }
    info->berr_unrefined = berr;

    // 4. iterative refinement (Sec. 5); a stalled or exhausted low-precision
    //    attempt re-solves with a double factorization of the same A~
    int iters = 0, attempt_iters = 0, gm_products = 0;
    double prev = berr;
    for (;;) {
        if (berr <= opts->tol) break;
        bool stalled = (attempt_iters > 0 && !(berr < 0.9 * prev)) || h_info >= 0;
        bool exhausted = attempt_iters >= opts->refine_max;
        if (stalled || exhausted) {
            if (cur_prec == RBT_F64 || !opts->fallback || !At64) break;
            // "responsibly reckless" fallback: refactor the same A~ in double;
            // a seven-digit sliced attempt first tries eight digits (the
            // pair copy fits the double buffer: both take 8 bytes an entry)
            const int next = cur_prec == RBT_DF64TC7 ? RBT_DF64TC : RBT_F64;
            fell_back = next == RBT_F64 ? 1 : 2;
            st = apply_2sided_wp(n, d, align, U, V, n, A, lda, At64, ldt, next, s, opts->kind);
            if (st != RBT_OK) return st;
            st = genp_factor(n, next, At64, ldt, d_info, fac, fac_bytes, 0, s);
            if (st != RBT_OK) return st;
            RBT_CUDA_TRY(cudaMemcpyAsync(&h_info, d_info, 8, cudaMemcpyDeviceToHost, s));
            RBT_CUDA_TRY(cudaStreamSynchronize(s));
            if (h_info == -2) return RBT_ERR_TIMEOUT;
            cur_prec = next;
            cur_At = At64;
            cur_ldt = ldt;
            attempt_iters = 0;
            prev = INFINITY;
            if (h_info >= 0) {
                if (next != RBT_F64) {
                    berr = INFINITY;  // a failed factor counts as a stall: on to double
                    continue;
                }
                rbt_status ps;
                st = read_pivot_status(h_info, RBT_F64, At64, ldt, s, &ps);
                if (st != RBT_OK) return st;
                info->status = ps;
                info->zero_pivot = h_info;
                info->fell_back = 1;
                info->iters = iters;
                return ps;
            }
            RBT_CUDA_TRY(cudaMemcpy2DAsync(X, ldx * 8, B, ldb * 8, n * 8, nrhs, cudaMemcpyDeviceToDevice, s));
            st = correction(n, nrhs, d, align, opts->kind, U, V, cur_prec, cur_At, cur_ldt, X, ldx, sol, sol_bytes, s);
            if (st != RBT_OK) return st;
            st = residual_impl(n, nrhs, A, lda, X, ldx, B, ldb, R, n, scal, scal + 1, res, s);
            if (st != RBT_OK) return st;
            RBT_CUDA_TRY(cudaMemcpyAsync(&berr, scal + 1, 8, cudaMemcpyDeviceToHost, s));
            RBT_CUDA_TRY(cudaStreamSynchronize(s));
            continue;
        }
        if (opts->refine_mode == RBT_REFINE_GMRES) {
            const int m = opts->restart > 0 ? opts->restart : kGmresDefaultRestart;
            int used = 0;
            for (int64_t c = 0; c < nrhs; c++) {
                st = gmres_cycle(n, d, align, opts->kind, U, V, cur_prec, cur_At, cur_ldt, sol, sol_bytes, A, lda, scal, res,
                                 R + c * n, X + c * ldx, m, w + L.gm, s, &used);
                if (st != RBT_OK) return st;
            }
            gm_products += used;
        } else {
            st = correction(n, nrhs, d, align, opts->kind, U, V, cur_prec, cur_At, cur_ldt, R, n, sol, sol_bytes, s);
            if (st != RBT_OK) return st;
            st = add_block(n, nrhs, R, n, X, ldx, s);
            if (st != RBT_OK) return st;
        }
        st = residual_impl(n, nrhs, A, lda, X, ldx, B, ldb, R, n, scal, scal + 1, res, s);
        if (st != RBT_OK) return st;
        prev = berr;
        RBT_CUDA_TRY(cudaMemcpyAsync(&berr, scal + 1, 8, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaMemcpyAsync(&h_wait, sol, 4, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_wait) return RBT_ERR_TIMEOUT;
        iters++;
        attempt_iters++;
    }
    // the last corrections of a fallback may not have been followed by a read
    RBT_CUDA_TRY(cudaMemcpyAsync(&h_wait, sol, 4, cudaMemcpyDeviceToHost, s));
    RBT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_wait) return RBT_ERR_TIMEOUT;
    info->iters = opts->refine_mode == RBT_REFINE_GMRES ? gm_products : iters;
    info->fell_back = fell_back;
    info->berr = berr;
    info->zero_pivot = -1;
    info->status = berr <= opts->tol ? RBT_OK : RBT_NOT_CONVERGED;
    return (rbt_status)info->status;
}

}  // extern "C"
