// Butterfly coefficient generator and the butterfly transforms (sm_103a).
//
// Two-sided transform A~ = U^T A V of Eq. (rbt-depth-d), fused over layers.
//
// Index structure.  With reference size m and half sizes h_k = m / 2^k, every
// butterfly of layer k pairs row i with row i + h_k.  For a run of layers
// k_lo..k_hi (L = k_hi - k_lo + 1 layers) write each row as
//     i = (c 2^L + s) h + r,   h = h_{k_hi},  r in [0, h),  s in [0, 2^L),
// so that layer k pairs local index s with s + 2^(k_hi - k) inside the group
// (c, r).  The 2^L x 2^L elements A[i_s, j_t] of a row group and a column
// group are therefore closed under all L layers on both sides: one thread
// loads them once, applies every layer in registers and stores them once.
// With k_lo = 1 and k_hi = d this is the single pass over the matrix that
// Sec. 3 proposes for small d (c = 0, h = m / 2^d = q).
//
// A butterfly pair (top s, bottom s + 2^l) exists when its bottom row is
// < n; a top row whose partner is past n is a nu row and passes through
// unscaled (Eq. O-matrix-definition).  The 1/sqrt(2) of each existing pair
// is applied together with the layer's random diagonal.
//
// Memory access: consecutive threads take consecutive r, so for every (s, t)
// a warp reads and writes 32 consecutive doubles of one column (256 B,
// coalesced), and each element crosses HBM exactly once per pass.
#include "common.cuh"
#include "df64.cuh"
#include "rbt_dev.cuh"

namespace rbt {

constexpr double kInvSqrt2 = 0.70710678118654752440084436210485;

// ------------------------------------------------------------ generator

__global__ void generate_kernel(int64_t n, int d, uint64_t seed, double *U, double *V, int64_t ldw)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t per_side = n * d;
    if (idx >= 2 * per_side) return;
    int side = idx >= per_side ? 1 : 0;
    int64_t rem = idx - side * per_side;
    int layer = (int)(rem / n) + 1;
    int64_t i = rem - (int64_t)(layer - 1) * n;
    (side ? V : U)[i + (int64_t)(layer - 1) * ldw] = coef_value(seed, side, layer, i);
}

// Packed coefficients of the rotation form (rot_value), same layout.
__global__ void generate_rot_kernel(int64_t n, int d, int64_t m, int ds, uint64_t seed, double *U, double *V,
                                    int64_t ldw)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t per_side = n * d;
    if (idx >= 2 * per_side) return;
    int side = idx >= per_side ? 1 : 0;
    int64_t rem = idx - side * per_side;
    int layer = (int)(rem / n) + 1;
    int64_t i = rem - (int64_t)(layer - 1) * n;
    (side ? V : U)[i + (int64_t)(layer - 1) * ldw] = rot_value(seed, side, layer, i, n, m, ds);
}

// ------------------------------------------------------ fused two-sided

template <typename T> __device__ __forceinline__ T cvt_out(double v);
template <> __device__ __forceinline__ double cvt_out<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt_out<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ df64 cvt_out<df64>(double v) { return df_from_double(v); }

constexpr int kTX = 128;  // threads per block along row groups

// One pass over layers k_hi .. k_hi-L+1 on both sides.  Layers pre_lo..pre_hi
// (diagonal only, k > d_s) are applied first when pre_hi >= pre_lo.
// ROT: the rotation form (R_k = I; each pair (a, b) with packed (c, s)
// becomes (c a + s b, s a - c b) on the rows with U's and on the columns
// with V's coefficients) instead of the scaled butterflies.
template <int L, typename TO, bool ROT = false>
__global__ void __launch_bounds__(kTX)
fused2_kernel(int64_t n, int64_t h, int64_t ngroups, int k_hi, int pre_lo, int pre_hi,
              const double *__restrict__ U, const double *__restrict__ V, int64_t ldw,
              const double *Ain, int64_t lda_in, TO *Aout, int64_t lda_out, int gpt)
{
    constexpr int G = 1 << L;
    const int64_t gr = blockIdx.x * (int64_t)kTX + threadIdx.x;
    if (gr >= ngroups) return;
    const int64_t cr = gr / h;
    const int64_t rr = gr - cr * h;

    int64_t row[G];
    bool rv[G];
#pragma unroll
    for (int s = 0; s < G; s++) {
        row[s] = (cr * G + s) * h + rr;
        rv[s] = row[s] < n;
    }
    // per-layer row factors: diagonal entry times 1/sqrt(2) when paired
    double fu[L][G];
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int k = k_hi - l;
        const int st = 1 << l;
#pragma unroll
        for (int s = 0; s < G; s++) {
            double u = rv[s] ? __ldg(U + row[s] + (int64_t)(k - 1) * ldw) : 0.0;
            fu[l][s] = (!ROT && rv[s | st]) ? u * kInvSqrt2 : u;
        }
    }
    double pu[G];
#pragma unroll
    for (int s = 0; s < G; s++) {
        double p = 1.0;
        for (int k = pre_lo; k <= pre_hi; k++)
            p *= rv[s] ? __ldg(U + row[s] + (int64_t)(k - 1) * ldw) : 0.0;
        pu[s] = p;
    }
    const bool has_pre = pre_hi >= pre_lo;

    const int64_t g0 = (int64_t)blockIdx.y * gpt;
    for (int it = 0; it < gpt; it++) {
        const int64_t gc = g0 + it;
        if (gc >= ngroups) break;
        const int64_t cc = gc / h;
        const int64_t rc = gc - cc * h;
        int64_t col[G];
        bool cv[G];
#pragma unroll
        for (int t = 0; t < G; t++) {
            col[t] = (cc * G + t) * h + rc;
            cv[t] = col[t] < n;
        }
        double x[G][G];
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++)
                x[s][t] = (rv[s] && cv[t]) ? Ain[row[s] + col[t] * lda_in] : 0.0;

        if (has_pre) {
#pragma unroll
            for (int t = 0; t < G; t++) {
                double p = 1.0;
                for (int k = pre_lo; k <= pre_hi; k++)
                    p *= cv[t] ? __ldg(V + col[t] + (int64_t)(k - 1) * ldw) : 0.0;
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] *= pu[s] * p;
            }
        }

#pragma unroll
        for (int l = 0; l < L; l++) {
            const int k = k_hi - l;
            const int st = 1 << l;
            if (ROT) {
#pragma unroll
                for (int s = 0; s < G; s++) {
                    if ((s & st) || !rv[s | st]) continue;
                    const double c = fu[l][s], sn = fu[l][s | st];
#pragma unroll
                    for (int t = 0; t < G; t++) {
                        const double a = x[s][t], b = x[s | st][t];
                        x[s][t] = c * a + sn * b;
                        x[s | st][t] = sn * a - c * b;
                    }
                }
                double fv[G];
#pragma unroll
                for (int t = 0; t < G; t++) fv[t] = cv[t] ? __ldg(V + col[t] + (int64_t)(k - 1) * ldw) : 0.0;
#pragma unroll
                for (int t = 0; t < G; t++) {
                    if ((t & st) || !cv[t | st]) continue;
                    const double c = fv[t], sn = fv[t | st];
#pragma unroll
                    for (int s = 0; s < G; s++) {
                        const double a = x[s][t], b = x[s][t | st];
                        x[s][t] = c * a + sn * b;
                        x[s][t | st] = sn * a - c * b;
                    }
                }
                continue;
            }
            // B_k on the rows
#pragma unroll
            for (int s = 0; s < G; s++) {
                if (s & st) continue;
                if (!rv[s | st]) continue;
#pragma unroll
                for (int t = 0; t < G; t++) {
                    double a = x[s][t], b = x[s | st][t];
                    x[s][t] = a + b;
                    x[s | st][t] = a - b;
                }
            }
            // B_k on the columns
#pragma unroll
            for (int t = 0; t < G; t++) {
                if (t & st) continue;
                if (!cv[t | st]) continue;
#pragma unroll
                for (int s = 0; s < G; s++) {
                    double a = x[s][t], b = x[s][t | st];
                    x[s][t] = a + b;
                    x[s][t | st] = a - b;
                }
            }
            // R_k, R'_k and the pair normalizations
#pragma unroll
            for (int t = 0; t < G; t++) {
                double v = cv[t] ? __ldg(V + col[t] + (int64_t)(k - 1) * ldw) : 0.0;
                double fv = cv[t | st] ? v * kInvSqrt2 : v;
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] = (x[s][t] * fu[l][s]) * fv;
            }
        }

#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++)
                if (rv[s] && cv[t]) Aout[row[s] + col[t] * lda_out] = cvt_out<TO>(x[s][t]);
    }
}

// n == 1 (no butterfly at all): out = in * prod U * prod V.
template <typename TO>
__global__ void diag_only_kernel(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                                 const double *Ain, int64_t lda_in, TO *Aout, int64_t lda_out)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    int64_t i = idx % n, j = idx / n;
    double p = Ain[i + j * lda_in];
    for (int k = 1; k <= d; k++) p *= U[i + (k - 1) * ldw] * V[j + (k - 1) * ldw];
    Aout[i + j * lda_out] = cvt_out<TO>(p);
}

template <typename TO>
static rbt_status transform2(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                             const double *Ain, int64_t lda_in, TO *Aout, int64_t lda_out, int max_l,
                             cudaStream_t stream, int64_t align = 1, bool rot = false);

// ------------------------------------------ float working copy, FP32 math

// double -> float, rounded to nearest even, from 32-bit integer operations on
// the two halves of the double, with no FP64-pipe instruction at all (the
// conversion instruction runs there, about two per clock per SM on this GPU;
// a rare-case branch to it would still be issued for every element once the
// compiler predicates it).  Truncated float bits = the exponent rebiased
// (- 896) and the top 23 mantissa bits (a funnel shift of the halves by 3);
// the 29 bits below them decide the rounding (up when above half, or at half
// with an odd last bit), the carry running into the exponent (to infinity
// past the largest float).  Outside the float normal range, by selects:
// signed zero below 2^-126 (results that would be subnormal flush to zero),
// infinity above, NaN kept NaN.
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned ex = (hi >> 20) & 0x7FFu;
    unsigned f = __funnelshift_l(lo, (hi & 0x7FFFFFFFu) - (896u << 20), 3);
    f += (lo << 3) > 0x80000000u - (f & 1u) ? 1u : 0u;
    f = ex < 897u ? 0u : f;
    const unsigned big = (ex == 2047u && ((hi & 0xFFFFFu) | lo) != 0u) ? 0x7FC00000u : 0x7F800000u;
    f = ex > 1150u ? big : f;
    return __uint_as_float(f | (hi & 0x80000000u));
}

// ------------------------------------ double-float working copy, FP32 math

// double -> float pair (hi + lo with |lo| <= ulp(hi) / 2, within 2^-48 |x|)
// by 32-bit integer operations on the halves of the double, no FP64-pipe
// instruction: hi is the double rounded to nearest even as in d2f_rn (with
// its zero / infinity / NaN selects); the remainder r below hi's last bit (the
// low 29 mantissa bits, less 2^29 when hi rounded up: |r| <= 2^28) goes
// through the integer-to-float unit and is scaled by the double's unit in the
// last place 2^(E - 1075).  Below |x| = 2^-74 that scale would leave the
// float normal range and lo is zero (hi alone, within 2^-24 |x| of x, a
// relative term far below the scale of any entry the transform mixes with).
__device__ __forceinline__ df64 split_double(double x)
{
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const unsigned ex = (hw >> 20) & 0x7FFu;
    unsigned f = __funnelshift_l(lw, (hw & 0x7FFFFFFFu) - (896u << 20), 3);
    const unsigned up = (lw << 3) > 0x80000000u - (f & 1u) ? 1u : 0u;
    f += up;
    f = ex < 897u ? 0u : f;
    const unsigned big = (ex == 2047u && ((hw & 0xFFFFFu) | lw) != 0u) ? 0x7FC00000u : 0x7F800000u;
    f = ex > 1150u ? big : f;
    const unsigned sign = hw & 0x80000000u;
    const float hi = __uint_as_float(f | sign);
    const int r = (int)(lw & 0x1FFFFFFFu) - (int)(up << 29);
    const float lo = (ex - 949u < 201u) ? __int2float_rn(r) * __int_as_float((int)(ex - 948u) << 23) : 0.f;
    return df64(hi, sign ? -lo : lo);
}

// Unnormalized double-float steps of the transform: a value is hi + lo with
// lo a few units in the last place of hi at most.  The leading parts add
// exactly (TwoSum), the trailing parts in float; products take the exact
// error of the leading product by FMA plus both cross terms.  No
// renormalization until the store: each step's error stays within about
// 2^-47 of the magnitudes it combines, the scale of the bounds the working
// copy is checked against.
__device__ __forceinline__ df64 lz_add(df64 a, df64 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df64(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 lz_sub(df64 a, df64 b) { return lz_add(a, df64(-b.hi, -b.lo)); }

__device__ __forceinline__ df64 lz_mul(df64 a, df64 c)
{
    const float p = __fmul_rn(a.hi, c.hi);
    float e = __fmaf_rn(a.hi, c.hi, -p);
    e = __fmaf_rn(a.hi, c.lo, e);
    e = __fmaf_rn(a.lo, c.hi, e);
    return df64(p, e);
}

// ------------------------------------------- pipelined working-copy pass
//
// The float and double-float working copies in one single pass over A, with
// the loads decoupled from the arithmetic: each thread's 2^L x 2^L group of
// the next column groups lands in shared memory by 8-byte cp.async (a
// leading dimension may be odd, so wider copies would not stay aligned) while
// the thread transforms the current one.  Each thread reads back only the
// slots it filled itself, so no barrier is needed after the first; the
// copies in flight per SM no longer depend on how many registers the
// arithmetic holds.
// Shape per layer count and output (F: the float copy), from sweeps on
// GB300 at n = 16384, 20001 (three layers), 40003 and 40960: threads per
// CTA, pipeline stages (copies run stages - 1 column groups ahead), column
// groups per CTA, and the CTAs per SM the register allocation must allow.
// Two layers: the float pass is fastest with the compiler's full register
// budget (3 CTAs per SM, 0.92 of HBM at n = 40003), the pair pass with at
// most 168 registers (3 CTAs; with 204 it fell from 0.60 to 0.52); a cap of
// 128 (4 CTAs) cost both (0.68, 0.52).  Three layers hold 64 entries a
// thread: few warps fit an SM, which bounds that pass.
template <int L, bool F> struct WpCfg {
    static constexpr int threads = (L == 3 && !F) ? 64 : 128;
    static constexpr int stages = L == 3 ? 2 : 3;
    static constexpr int gpt = (L == 3 && !F) ? 8 : 16;        // column groups per CTA
    static constexpr int min_blocks = (L == 2 && !F) ? 3 : 1;
};

__device__ __forceinline__ void cp_async8z(double *smem, const double *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The arithmetic of each working precision: float (from the double input by
// d2f_rn), or unnormalized double-float pairs (split_double, lz_*).
struct WpFloat {
    using T = float;
    static __device__ __forceinline__ T cvt(double x) { return d2f_rn(x); }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T one() { return 1.f; }
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ T inv_sqrt2() { return 0.70710678118654752440f; }
    static __device__ __forceinline__ void store(float *p, T v) { __stcs(p, v); }
};

struct WpPair {
    using T = df64;
    static __device__ __forceinline__ T cvt(double x) { return split_double(x); }
    static __device__ __forceinline__ T add(T a, T b) { return lz_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return lz_sub(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return lz_mul(a, b); }
    static __device__ __forceinline__ T one() { return df64(1.f); }
    static __device__ __forceinline__ T zero() { return df64(0.f); }
    static __device__ __forceinline__ T inv_sqrt2()
    {
        constexpr double kSd = 0.70710678118654752440;
        constexpr float kSh = (float)kSd;
        return df64(kSh, (float)(kSd - (double)kSh));
    }
    static __device__ __forceinline__ void store(df64 *p, T v)
    {
        float hs, ls;
        two_sum(v.hi, v.lo, hs, ls);  // the leading part may have cancelled: renormalize once
        __stcs(reinterpret_cast<float2 *>(p), make_float2(hs, ls));
    }
};

// Single pass of layers k_hi = d_s .. 1 (row i = s h + r, s < 2^L, h = m / 2^L),
// diagonal-only layers pre_lo .. pre_hi first; output element type OUT.
template <int L, class W, typename OUT, bool ROT>
__global__ void __launch_bounds__(WpCfg<L, sizeof(OUT) == 4>::threads, WpCfg<L, sizeof(OUT) == 4>::min_blocks)
fused2_wp_kernel(int64_t n, int64_t h, int k_hi, int pre_lo, int pre_hi, const double *__restrict__ U,
                 const double *__restrict__ V, int64_t ldw, const double *__restrict__ Ain, int64_t lda_in,
                 OUT *__restrict__ Aout, int64_t lda_out)
{
    using T = typename W::T;
    constexpr int G = 1 << L, E = G * G;
    using C = WpCfg<L, sizeof(OUT) == 4>;
    constexpr int NT = C::threads, ST = C::stages, GPT = C::gpt;
    static_assert(GPT * G <= NT, "one thread per column coefficient");
    extern __shared__ __align__(16) double wp_smem[];               // [ST][E][NT] landing slots
    __shared__ T s_fv[GPT][L][G], s_pv[GPT][G];                     // column factors per group
    __shared__ bool s_cv[GPT][G];
    const int tid = threadIdx.x;
    const int64_t gc0 = (int64_t)blockIdx.y * GPT;
    const int ng = (int)(h - gc0 < GPT ? h - gc0 : GPT);
    if (tid < GPT * G) {
        const int it = tid / G, t = tid % G;
        const int64_t gc = gc0 + it;
        bool ok = false;
        T p = W::one();
        if (it < ng) {
            const int64_t c = t * h + gc;
            ok = c < n;
            for (int k = pre_lo; k <= pre_hi; k++) p = W::mul(p, ok ? W::cvt(__ldg(V + c + (int64_t)(k - 1) * ldw)) : W::zero());
#pragma unroll
            for (int l = 0; l < L; l++) {
                const int k = k_hi - l, st = 1 << l;
                const int64_t cp = (t | st) * h + gc;  // the partner column of this layer
                const T v = ok ? W::cvt(__ldg(V + c + (int64_t)(k - 1) * ldw)) : W::zero();
                s_fv[it][l][t] = (!ROT && cp < n) ? W::mul(v, W::inv_sqrt2()) : v;
            }
        } else {
#pragma unroll
            for (int l = 0; l < L; l++) s_fv[it][l][t] = W::zero();
        }
        s_pv[it][t] = p;
        s_cv[it][t] = ok;
    }
    __syncthreads();
    const int64_t rr = blockIdx.x * (int64_t)NT + tid;
    if (rr >= h) return;
    int64_t row[G];
    bool rv[G];
#pragma unroll
    for (int s = 0; s < G; s++) {
        row[s] = s * h + rr;
        rv[s] = row[s] < n;
    }
    double *slot = wp_smem + tid;
    auto issue = [&](int it) {
        if (it < ng) {
            double *dst = slot + (it % ST) * E * NT;
#pragma unroll
            for (int t = 0; t < G; t++) {
                const bool okt = s_cv[it][t];
                const double *colp = Ain + (t * h + gc0 + it) * lda_in;
#pragma unroll
                for (int s = 0; s < G; s++) {
                    const bool ok = okt && rv[s];
                    cp_async8z(dst + (t * G + s) * NT, ok ? colp + row[s] : Ain, ok);
                }
            }
        }
        cp_async_commit_group();
    };
#pragma unroll
    for (int i = 0; i < ST - 1; i++) issue(i);
    // row factors (layers, and the product of the diagonal-only layers)
    T fu[L][G], pu[G];
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int k = k_hi - l, st = 1 << l;
#pragma unroll
        for (int s = 0; s < G; s++) {
            const T u = rv[s] ? W::cvt(__ldg(U + row[s] + (int64_t)(k - 1) * ldw)) : W::zero();
            fu[l][s] = (!ROT && rv[s | st]) ? W::mul(u, W::inv_sqrt2()) : u;
        }
    }
    const bool has_pre = pre_hi >= pre_lo;
#pragma unroll
    for (int s = 0; s < G; s++) {
        T p = W::one();
        for (int k = pre_lo; k <= pre_hi; k++) p = W::mul(p, rv[s] ? W::cvt(__ldg(U + row[s] + (int64_t)(k - 1) * ldw)) : W::zero());
        pu[s] = p;
    }
    for (int it = 0; it < ng; it++) {
        issue(it + ST - 1);
        cp_async_wait_group<ST - 1>();  // this thread's copies of group it have landed
        const double *src = slot + (it % ST) * E * NT;
        T x[G][G];
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++) x[s][t] = W::cvt(src[(t * G + s) * NT]);
        if (has_pre) {
#pragma unroll
            for (int t = 0; t < G; t++) {
                const T p = s_pv[it][t];
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] = W::mul(x[s][t], W::mul(pu[s], p));
            }
        }
#pragma unroll
        for (int l = 0; l < L; l++) {
            const int st = 1 << l;
            if (ROT) {
#pragma unroll
                for (int s = 0; s < G; s++) {
                    if ((s & st) || !rv[s | st]) continue;
                    const T c = fu[l][s], sn = fu[l][s | st];
#pragma unroll
                    for (int t = 0; t < G; t++) {
                        const T p = x[s][t], q = x[s | st][t];
                        x[s][t] = W::add(W::mul(c, p), W::mul(sn, q));
                        x[s | st][t] = W::sub(W::mul(sn, p), W::mul(c, q));
                    }
                }
#pragma unroll
                for (int t = 0; t < G; t++) {
                    if ((t & st) || !s_cv[it][t | st]) continue;
                    const T c = s_fv[it][l][t], sn = s_fv[it][l][t | st];
#pragma unroll
                    for (int s = 0; s < G; s++) {
                        const T p = x[s][t], q = x[s][t | st];
                        x[s][t] = W::add(W::mul(c, p), W::mul(sn, q));
                        x[s][t | st] = W::sub(W::mul(sn, p), W::mul(c, q));
                    }
                }
                continue;
            }
#pragma unroll
            for (int s = 0; s < G; s++) {
                if ((s & st) || !rv[s | st]) continue;
#pragma unroll
                for (int t = 0; t < G; t++) {
                    const T p = x[s][t], q = x[s | st][t];
                    x[s][t] = W::add(p, q);
                    x[s | st][t] = W::sub(p, q);
                }
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                if ((t & st) || !s_cv[it][t | st]) continue;
#pragma unroll
                for (int s = 0; s < G; s++) {
                    const T p = x[s][t], q = x[s][t | st];
                    x[s][t] = W::add(p, q);
                    x[s][t | st] = W::sub(p, q);
                }
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                const T fv = s_fv[it][l][t];
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] = W::mul(W::mul(x[s][t], fu[l][s]), fv);
            }
        }
        const int64_t gc = gc0 + it;
#pragma unroll
        for (int t = 0; t < G; t++) {
            if (!s_cv[it][t]) continue;
            OUT *colp = Aout + (t * h + gc) * lda_out;
#pragma unroll
            for (int s = 0; s < G; s++)
                if (rv[s]) W::store(colp + row[s], x[s][t]);
        }
    }
    cp_async_wait_group<0>();
}

// Launch of the pipelined pass for d_s = L layers (1 .. 3), either kind.
template <int L, class W, typename OUT>
static rbt_status launch_wp(int64_t n, int64_t h, int ds, int d, const double *U, const double *V, int64_t ldw,
                            const double *Ain, int64_t lda_in, OUT *Aout, int64_t lda_out, bool rot,
                            cudaStream_t stream)
{
    using C = WpCfg<L, sizeof(OUT) == 4>;
    constexpr int NT = C::threads, ST = C::stages, GPT = C::gpt;
    constexpr int smem = ST * (1 << (2 * L)) * NT * (int)sizeof(double);
    static PerDeviceOnce once, once_rot;
    rbt_status st = rot ? smem_opt_in(once_rot, fused2_wp_kernel<L, W, OUT, true>, smem)
                        : smem_opt_in(once, fused2_wp_kernel<L, W, OUT, false>, smem);
    if (st != RBT_OK) return st;
    dim3 grid((unsigned)cdiv(h, NT), (unsigned)cdiv(h, GPT));
    if (rot)
        fused2_wp_kernel<L, W, OUT, true><<<grid, NT, smem, stream>>>(n, h, ds, ds + 1, d, U, V, ldw, Ain, lda_in,
                                                                       Aout, lda_out);
    else
        fused2_wp_kernel<L, W, OUT, false><<<grid, NT, smem, stream>>>(n, h, ds, ds + 1, d, U, V, ldw, Ain, lda_in,
                                                                        Aout, lda_out);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

template <class W, typename OUT>
static rbt_status transform_wp(int64_t n, int d, const double *U, const double *V, int64_t ldw, const double *Ain,
                               int64_t lda_in, OUT *Aout, int64_t lda_out, cudaStream_t stream, int64_t align, bool rot)
{
    const int ds = eff_depth(n, d);
    ProfScope ps(kProfTransform, stream);
    const int64_t h = ref_size(n, d, align) >> ds;
    switch (ds) {
    case 1: return launch_wp<1, W, OUT>(n, h, ds, d, U, V, ldw, Ain, lda_in, Aout, lda_out, rot, stream);
    case 2: return launch_wp<2, W, OUT>(n, h, ds, d, U, V, ldw, Ain, lda_in, Aout, lda_out, rot, stream);
    default: return launch_wp<3, W, OUT>(n, h, ds, d, U, V, ldw, Ain, lda_in, Aout, lda_out, rot, stream);
    }
}

// The working copies of the float-storage and double-float precisions: one
// pipelined pass for d_s <= 3 (float arithmetic for the float copy,
// unnormalized double-float arithmetic on the FP32 pipes for the pair copy;
// refinement always measures against A in double); deeper transforms take the
// double passes of transform2 and round at the end.
static rbt_status transform2_f32math(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                                     const double *Ain, int64_t lda_in, float *Aout, int64_t lda_out,
                                     cudaStream_t stream, int64_t align = 1, bool rot = false)
{
    const int ds = eff_depth(n, d);
    if (ds == 0 || ds > 3)
        return transform2<float>(n, d, U, V, ldw, Ain, lda_in, Aout, lda_out, 3, stream, align, rot);
    return transform_wp<WpFloat, float>(n, d, U, V, ldw, Ain, lda_in, Aout, lda_out, stream, align, rot);
}

static rbt_status transform2_df64math(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                                      const double *Ain, int64_t lda_in, df64 *Aout, int64_t lda_out,
                                      cudaStream_t stream, int64_t align = 1, bool rot = false)
{
    const int ds = eff_depth(n, d);
    if (ds == 0 || ds > 3)
        return transform2<df64>(n, d, U, V, ldw, Ain, lda_in, Aout, lda_out, 3, stream, align, rot);
    return transform_wp<WpPair, df64>(n, d, U, V, ldw, Ain, lda_in, Aout, lda_out, stream, align, rot);
}

template <int L, typename TO>
static void launch_fused2(int64_t n, int64_t h, int64_t ngroups, int k_hi, int pre_lo, int pre_hi,
                          const double *U, const double *V, int64_t ldw, const double *Ain,
                          int64_t lda_in, TO *Aout, int64_t lda_out, cudaStream_t stream, bool rot)
{
    const int gpt = 4;
    dim3 grid((unsigned)cdiv(ngroups, kTX), (unsigned)cdiv(ngroups, gpt));
    if (rot)
        fused2_kernel<L, TO, true><<<grid, kTX, 0, stream>>>(n, h, ngroups, k_hi, pre_lo, pre_hi, U, V, ldw, Ain,
                                                             lda_in, Aout, lda_out, gpt);
    else
        fused2_kernel<L, TO, false><<<grid, kTX, 0, stream>>>(n, h, ngroups, k_hi, pre_lo, pre_hi, U, V, ldw, Ain,
                                                              lda_in, Aout, lda_out, gpt);
}

// Run layers in passes of at most max_l layers, from layer d_s down to 1.
template <typename TO>
static rbt_status transform2(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                             const double *Ain, int64_t lda_in, TO *Aout, int64_t lda_out, int max_l,
                             cudaStream_t stream, int64_t align, bool rot)
{
    if (n == 0) return RBT_OK;
    ProfScope ps(kProfTransform, stream);
    const int ds = eff_depth(n, d);
    const int64_t m = ref_size(n, d, align);
    if (ds == 0) {
        int64_t tot = n * n;
        diag_only_kernel<TO><<<(unsigned)cdiv(tot, 256), 256, 0, stream>>>(n, d, U, V, ldw, Ain, lda_in,
                                                                            Aout, lda_out);
        RBT_LAUNCH_CHECK();
        return RBT_OK;
    }
    int k_hi = ds;
    bool first = true;
    const double *src = Ain;
    int64_t ld_src = lda_in;
    while (k_hi >= 1) {
        int L = k_hi < max_l ? k_hi : max_l;
        int k_lo = k_hi - L + 1;
        int64_t h = m >> k_hi;
        int64_t ngroups = ((int64_t)1 << (k_lo - 1)) * h;
        int pre_lo = first ? ds + 1 : 1, pre_hi = first ? d : 0;
        bool last = (k_lo == 1);
        // intermediate passes stay in double inside Aout when it is double;
        // a float output is only written by the last pass (max_l covers d_s).
        if (!last && sizeof(TO) != sizeof(double)) return RBT_ERR_UNSUPPORTED;
        TO *dst = Aout;
        switch (L) {
        case 1: launch_fused2<1, TO>(n, h, ngroups, k_hi, pre_lo, pre_hi, U, V, ldw, src, ld_src, dst, lda_out, stream, rot); break;
        case 2: launch_fused2<2, TO>(n, h, ngroups, k_hi, pre_lo, pre_hi, U, V, ldw, src, ld_src, dst, lda_out, stream, rot); break;
        default: launch_fused2<3, TO>(n, h, ngroups, k_hi, pre_lo, pre_hi, U, V, ldw, src, ld_src, dst, lda_out, stream, rot); break;
        }
        RBT_LAUNCH_CHECK();
        src = reinterpret_cast<const double *>(Aout);
        ld_src = lda_out;
        first = false;
        k_hi = k_lo - 1;
    }
    return RBT_OK;
}

// ------------------------------------------------------- one-sided

// trans = 1: B <- W^T B: layers k = d..1, each B_k then R_k.
// trans = 0: B <- W B:   layers k = 1..d, each R_k then B_k.
// One pass covers layers k_lo..k_hi; extra diagonal-only layers (k > d_s)
// are folded in as `ext` (before the pass for trans = 1, after it for 0).
template <int L, bool ROT>
__global__ void __launch_bounds__(kTX)
vec_kernel(int64_t n, int64_t h, int64_t ngroups, int k_hi, int trans, int ext_lo, int ext_hi,
           const double *__restrict__ W, int64_t ldw, double *B, int64_t ldb)
{
    const int64_t gr = blockIdx.x * (int64_t)kTX + threadIdx.x;
    if (gr >= ngroups) return;
    vec_group<L, ROT>(n, h, k_hi, trans, ext_lo, ext_hi, W, ldw, B + (int64_t)blockIdx.y * ldb, gr);
}

__global__ void vec_diag_only_kernel(int64_t n, int d, const double *W, int64_t ldw, double *B,
                                     int64_t ldb, int64_t nrhs)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t i = idx % n, c = idx / n;
    double p = B[i + c * ldb];
    for (int k = 1; k <= d; k++) p *= W[i + (k - 1) * ldw];
    B[i + c * ldb] = p;
}

template <int L>
static void launch_vec(int64_t n, int64_t h, int64_t ngroups, int k_hi, int trans, int ext_lo, int ext_hi,
                       const double *W, int64_t ldw, double *B, int64_t ldb, int64_t nrhs,
                       cudaStream_t stream, bool rot)
{
    dim3 grid((unsigned)cdiv(ngroups, kTX), (unsigned)nrhs);
    if (rot)
        vec_kernel<L, true><<<grid, kTX, 0, stream>>>(n, h, ngroups, k_hi, trans, ext_lo, ext_hi, W, ldw, B, ldb);
    else
        vec_kernel<L, false><<<grid, kTX, 0, stream>>>(n, h, ngroups, k_hi, trans, ext_lo, ext_hi, W, ldw, B, ldb);
}

static rbt_status vec_transform(int64_t n, int d, const double *W, int64_t ldw, int trans, double *B,
                                int64_t ldb, int64_t nrhs, cudaStream_t stream, int64_t align = 1, bool rot = false)
{
    if (n == 0 || nrhs == 0) return RBT_OK;
    const int ds = eff_depth(n, d);
    const int64_t m = ref_size(n, d, align);
    if (ds == 0) {
        vec_diag_only_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, d, W, ldw, B, ldb, nrhs);
        RBT_LAUNCH_CHECK();
        return RBT_OK;
    }
    // chunk boundaries, from the top layer down: [k_hi .. k_lo]
    int his[64], los[64], nch = 0;
    for (int k_hi = ds; k_hi >= 1;) {
        int L = k_hi < 3 ? k_hi : 3;
        his[nch] = k_hi;
        los[nch] = k_hi - L + 1;
        nch++;
        k_hi -= L;
    }
    for (int ci = 0; ci < nch; ci++) {
        int idx = trans ? ci : (nch - 1 - ci);
        int k_hi = his[idx], k_lo = los[idx];
        int L = k_hi - k_lo + 1;
        int64_t h = m >> k_hi;
        int64_t ngroups = ((int64_t)1 << (k_lo - 1)) * h;
        // extra diagonal-only layers: first pass of trans, last pass of !trans
        bool with_ext = trans ? (ci == 0) : (ci == nch - 1);
        int ext_lo = with_ext ? ds + 1 : 1, ext_hi = with_ext ? d : 0;
        for (int64_t c0 = 0; c0 < nrhs; c0 += 65535) {
            int64_t nc = nrhs - c0 < 65535 ? nrhs - c0 : 65535;
            double *Bc = B + c0 * ldb;
            switch (L) {
            case 1: launch_vec<1>(n, h, ngroups, k_hi, trans, ext_lo, ext_hi, W, ldw, Bc, ldb, nc, stream, rot); break;
            case 2: launch_vec<2>(n, h, ngroups, k_hi, trans, ext_lo, ext_hi, W, ldw, Bc, ldb, nc, stream, rot); break;
            default: launch_vec<3>(n, h, ngroups, k_hi, trans, ext_lo, ext_hi, W, ldw, Bc, ldb, nc, stream, rot); break;
            }
            RBT_LAUNCH_CHECK();
        }
    }
    return RBT_OK;
}

int device_sm_count()
{
    // cached per device (up to 64 devices; others are queried every time)
    static std::atomic<int> cached[64];
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return kNumSMs;
    if (dev >= 0 && dev < 64 && (v = cached[dev].load(std::memory_order_relaxed)) > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return kNumSMs;
    if (dev >= 0 && dev < 64) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

}  // namespace rbt

using namespace rbt;

static bool overlap_bad(const void *a, int64_t lda, const void *b, int64_t ldb, int64_t n, size_t es_a,
                        size_t es_b)
{
    if (n == 0) return false;
    const char *a0 = (const char *)a, *b0 = (const char *)b;
    const char *a1 = a0 + ((size_t)(n - 1) * lda + n) * es_a;
    const char *b1 = b0 + ((size_t)(n - 1) * ldb + n) * es_b;
    bool disjoint = a1 <= b0 || b1 <= a0;
    bool same = (a0 == b0) && (lda == ldb) && (es_a == es_b);
    return !(disjoint || same);
}

extern "C" {

const char *rbt_status_string(int status)
{
    switch (status) {
    case RBT_OK: return "ok";
    case RBT_ERR_ARG: return "invalid argument";
    case RBT_ERR_CUDA: return "CUDA error";
    case RBT_ERR_WORKSPACE: return "workspace too small";
    case RBT_ERR_TIMEOUT: return "device wait timed out";
    case RBT_ERR_UNSUPPORTED: return "unsupported request";
    case RBT_ZERO_PIVOT: return "zero pivot";
    case RBT_NONFINITE: return "non-finite pivot";
    case RBT_NOT_CONVERGED: return "refinement did not converge";
    default: return "unknown status";
    }
}

int64_t rbt_reference_size(int64_t n, int32_t d, int64_t align, int32_t grid_p, int32_t grid_q)
{
    if (n < 0 || d < 0 || d > 62 || align < 0) return -1;
    if (grid_p < 0 || grid_q < 0 || grid_p > kMaxGridSide || grid_q > kMaxGridSide) return -1;
    const int64_t l = lcm_i64(grid_p > 1 ? grid_p : 1, grid_q > 1 ? grid_q : 1);  // <= 2^24
    const int64_t a0 = align > 1 ? align : 1;
    if (a0 > ((int64_t)1 << 62) / l) return -1;
    const int64_t a = a0 * l;                                                     // <= 2^62
    const int ds = eff_depth(n, d);
    if (a > (((int64_t)1 << 62) >> ds)) return -1;
    const int64_t p = a << ds;                                                    // <= 2^62
    const int64_t c = n / p + (n % p != 0 ? 1 : 0);
    if (c > 0 && p > INT64_MAX / c) return -1;
    return p * c;
}

rbt_status rbt_generate(int64_t n, int32_t d, uint64_t seed, double *U, double *V, int64_t ldw,
                        cudaStream_t stream)
{
    if (n < 0 || d < 0 || ldw < (n > 1 ? n : 1)) return RBT_ERR_ARG;
    if (n == 0 || d == 0) return RBT_OK;
    if (!U || !V) return RBT_ERR_ARG;
    int64_t tot = 2 * n * (int64_t)d;
    generate_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, stream>>>(n, d, seed, U, V, ldw);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status rbt_generate_rot(int64_t n, int32_t d, int64_t align, uint64_t seed, double *U, double *V, int64_t ldw,
                            cudaStream_t stream)
{
    if (n < 0 || d < 0 || d > 62 || align < 0 || ldw < (n > 1 ? n : 1)) return RBT_ERR_ARG;
    if (n == 0 || d == 0) return RBT_OK;
    if (!U || !V) return RBT_ERR_ARG;
    int64_t tot = 2 * n * (int64_t)d;
    generate_rot_kernel<<<(unsigned)cdiv(tot, 256), 256, 0, stream>>>(n, d, ref_size(n, d, align), eff_depth(n, d),
                                                                       seed, U, V, ldw);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

static rbt_status apply_2sided_f64(int64_t n, int32_t d, int64_t align, bool rot, const double *U, const double *V,
                                   int64_t ldw, const double *A_in, int64_t lda_in, double *A_out, int64_t lda_out,
                                   cudaStream_t stream)
{
    if (n < 0 || d < 0 || d > 62 || align < 0) return RBT_ERR_ARG;
    int64_t mn = n > 1 ? n : 1;
    if (lda_in < mn || lda_out < mn || (d > 0 && ldw < mn)) return RBT_ERR_ARG;
    if (n == 0) return RBT_OK;
    if (!A_in || !A_out || (d > 0 && (!U || !V))) return RBT_ERR_ARG;
    if (overlap_bad(A_in, lda_in, A_out, lda_out, n, 8, 8)) return RBT_ERR_ARG;
    if (d == 0) {
        if (A_in != A_out)
            RBT_CUDA_TRY(cudaMemcpy2DAsync(A_out, lda_out * 8, A_in, lda_in * 8, n * 8, n,
                                           cudaMemcpyDeviceToDevice, stream));
        return RBT_OK;
    }
    return transform2<double>(n, d, U, V, ldw, A_in, lda_in, A_out, lda_out, 3, stream, align, rot);
}

rbt_status rbt_apply_2sided_tiled(int64_t n, int32_t d, int64_t align, const double *U, const double *V,
                                  int64_t ldw, const double *A_in, int64_t lda_in, double *A_out, int64_t lda_out,
                                  cudaStream_t stream)
{
    return apply_2sided_f64(n, d, align, false, U, V, ldw, A_in, lda_in, A_out, lda_out, stream);
}

rbt_status rbt_apply_2sided(int64_t n, int32_t d, const double *U, const double *V, int64_t ldw,
                            const double *A_in, int64_t lda_in, double *A_out, int64_t lda_out,
                            cudaStream_t stream)
{
    return rbt_apply_2sided_tiled(n, d, 1, U, V, ldw, A_in, lda_in, A_out, lda_out, stream);
}

}  // extern "C"

namespace rbt {

rbt_status apply_2sided_wp(int64_t n, int32_t d, int64_t align, const double *U, const double *V, int64_t ldw,
                           const double *A_in, int64_t lda_in, void *A_out, int64_t lda_out, int32_t prec,
                           cudaStream_t stream, int32_t kind)
{
    if (n < 0 || d < 0 || d > 62 || align < 0 || prec < RBT_F64 || prec > kLastPrec) return RBT_ERR_ARG;
    if (kind != RBT_KIND_SCALED && kind != RBT_KIND_ROTATION) return RBT_ERR_ARG;
    const bool rot = kind == RBT_KIND_ROTATION;
    int64_t mn = n > 1 ? n : 1;
    if (lda_in < mn || lda_out < mn || (d > 0 && ldw < mn)) return RBT_ERR_ARG;
    if (n == 0) return RBT_OK;
    if (!A_in || !A_out || (d > 0 && (!U || !V))) return RBT_ERR_ARG;
    size_t es = prec == RBT_F64 || is_df64_storage(prec) ? 8 : 4;
    if ((const void *)A_in == A_out || overlap_bad(A_in, lda_in, A_out, lda_out, n, 8, es)) return RBT_ERR_ARG;
    if (prec == RBT_F64)
        return apply_2sided_f64(n, d, align, rot, U, V, ldw, A_in, lda_in, (double *)A_out, lda_out, stream);
    if (eff_depth(n, d) > 3) return RBT_ERR_UNSUPPORTED;  // one pass must cover every layer
    if (is_df64_storage(prec))
        return transform2_df64math(n, d, U, V, ldw, A_in, lda_in, (df64 *)A_out, lda_out, stream, align, rot);
    return transform2_f32math(n, d, U, V, ldw, A_in, lda_in, (float *)A_out, lda_out, stream, align, rot);
}

rbt_status apply_vec(int64_t n, int32_t d, int64_t align, const double *W, int64_t ldw, int32_t trans,
                     double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream, int32_t kind)
{
    if (n < 0 || d < 0 || d > 62 || nrhs < 0 || align < 0) return RBT_ERR_ARG;
    if (kind != RBT_KIND_SCALED && kind != RBT_KIND_ROTATION) return RBT_ERR_ARG;
    int64_t mn = n > 1 ? n : 1;
    if (ldb < mn || (d > 0 && ldw < mn)) return RBT_ERR_ARG;
    if (n == 0 || nrhs == 0 || d == 0) return RBT_OK;
    if (!W || !B) return RBT_ERR_ARG;
    return vec_transform(n, d, W, ldw, trans ? 1 : 0, B, ldb, nrhs, stream, align, kind == RBT_KIND_ROTATION);
}

}  // namespace rbt

extern "C" {

rbt_status rbt_apply_2sided_wp(int64_t n, int32_t d, const double *U, const double *V, int64_t ldw,
                               const double *A_in, int64_t lda_in, void *A_out, int64_t lda_out, int32_t prec,
                               cudaStream_t stream)
{
    return rbt::apply_2sided_wp(n, d, 1, U, V, ldw, A_in, lda_in, A_out, lda_out, prec, stream, RBT_KIND_SCALED);
}

rbt_status rbt_apply_2sided_layered(int64_t n, int32_t d, const double *U, const double *V,
                                    int64_t ldw, double *A, int64_t lda, cudaStream_t stream)
{
    if (n < 0 || d < 0 || d > 62) return RBT_ERR_ARG;
    int64_t mn = n > 1 ? n : 1;
    if (lda < mn || (d > 0 && ldw < mn)) return RBT_ERR_ARG;
    if (n == 0 || d == 0) return RBT_OK;
    if (!A || !U || !V) return RBT_ERR_ARG;
    return transform2<double>(n, d, U, V, ldw, A, lda, A, lda, 1, stream);
}

rbt_status rbt_apply_vec(int64_t n, int32_t d, const double *W, int64_t ldw, int32_t trans, double *B,
                         int64_t ldb, int64_t nrhs, cudaStream_t stream)
{
    return rbt::apply_vec(n, d, 1, W, ldw, trans, B, ldb, nrhs, stream, RBT_KIND_SCALED);
}

rbt_status rbt_apply_vec_tiled(int64_t n, int32_t d, int64_t align, const double *W, int64_t ldw, int32_t trans,
                               double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream)
{
    return rbt::apply_vec(n, d, align, W, ldw, trans, B, ldb, nrhs, stream, RBT_KIND_SCALED);
}

rbt_status rbt_transform_2sided(int64_t n, int32_t d, int64_t align, int32_t kind, int32_t prec, const double *U,
                                const double *V, int64_t ldw, const double *A_in, int64_t lda_in, void *A_out,
                                int64_t lda_out, cudaStream_t stream)
{
    if (prec == RBT_F64) {
        if (kind != RBT_KIND_SCALED && kind != RBT_KIND_ROTATION) return RBT_ERR_ARG;
        return apply_2sided_f64(n, d, align, kind == RBT_KIND_ROTATION, U, V, ldw, A_in, lda_in, (double *)A_out,
                                lda_out, stream);
    }
    return rbt::apply_2sided_wp(n, d, align, U, V, ldw, A_in, lda_in, A_out, lda_out, prec, stream, kind);
}

rbt_status rbt_transform_vec(int64_t n, int32_t d, int64_t align, int32_t kind, const double *W, int64_t ldw,
                             int32_t trans, double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream)
{
    return rbt::apply_vec(n, d, align, W, ldw, trans, B, ldb, nrhs, stream, kind);
}

}  // extern "C"
