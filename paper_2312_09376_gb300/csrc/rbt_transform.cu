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

// The working copy of the float-factor precisions only needs float accuracy
// (refinement always measures against A in double), so this pass reads A in
// double, converts once, and runs every layer in FP32: it is HBM-bound
// (12 bytes per entry) where the double-arithmetic pass is FP64-ALU bound.
constexpr int kF32Gpt = 2;  // column groups per thread of the float pass

template <int L, bool ROT = false>
__global__ void __launch_bounds__(kTX)
fused2_f32_kernel(int64_t n, int64_t h, int64_t ngroups, int k_hi, int pre_lo, int pre_hi,
                  const double *__restrict__ U, const double *__restrict__ V, int64_t ldw,
                  const double *__restrict__ Ain, int64_t lda_in, float *__restrict__ Aout, int64_t lda_out, int gpt)
{
    constexpr int G = 1 << L;
    constexpr float kS = 0.70710678118654752440f;
    // The column groups of this CTA are the same for all its threads: their
    // coefficients are converted once, into shared memory (each conversion
    // from double is an FP64-pipe instruction, the pass's scarce resource).
    __shared__ float sfv[kF32Gpt][L][G], spv[kF32Gpt][G];
    __shared__ bool scv[kF32Gpt][G];
    if ((int)threadIdx.x < gpt * G) {
        const int it = threadIdx.x / G, t = threadIdx.x % G;
        const int64_t gc = (int64_t)blockIdx.y * gpt + it;
        bool ok = false;
        float p = 0.f;
        if (gc < ngroups) {
            const int64_t cc = gc / h, rc = gc - cc * h;
            const int64_t c = (cc * G + t) * h + rc;
            ok = c < n;
            p = 1.f;
            for (int k = pre_lo; k <= pre_hi; k++) p *= ok ? __double2float_rn(__ldg(V + c + (int64_t)(k - 1) * ldw)) : 0.f;
#pragma unroll
            for (int l = 0; l < L; l++) {
                const int k = k_hi - l, st = 1 << l;
                const int64_t cp = (cc * G + (t | st)) * h + rc;  // the partner column of this layer
                const float v = ok ? __double2float_rn(__ldg(V + c + (int64_t)(k - 1) * ldw)) : 0.f;
                sfv[it][l][t] = (!ROT && cp < n) ? v * kS : v;
            }
        } else {
#pragma unroll
            for (int l = 0; l < L; l++) sfv[it][l][t] = 0.f;
        }
        spv[it][t] = p;
        scv[it][t] = ok;
    }
    __syncthreads();
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
    float fu[L][G], pu[G];
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int k = k_hi - l;
        const int st = 1 << l;
#pragma unroll
        for (int s = 0; s < G; s++) {
            float u = rv[s] ? __double2float_rn(__ldg(U + row[s] + (int64_t)(k - 1) * ldw)) : 0.f;
            fu[l][s] = (!ROT && rv[s | st]) ? u * kS : u;
        }
    }
#pragma unroll
    for (int s = 0; s < G; s++) {
        float p = 1.f;
        for (int k = pre_lo; k <= pre_hi; k++) p *= rv[s] ? __double2float_rn(__ldg(U + row[s] + (int64_t)(k - 1) * ldw)) : 0.f;
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
            cv[t] = scv[it][t];
        }
        float x[G][G];
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++)
                x[s][t] = (rv[s] && cv[t]) ? __double2float_rn(__ldcs(Ain + row[s] + col[t] * lda_in)) : 0.f;
        if (has_pre) {
#pragma unroll
            for (int t = 0; t < G; t++) {
                const float p = spv[it][t];
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
                    const float c = fu[l][s], sn = fu[l][s | st];
#pragma unroll
                    for (int t = 0; t < G; t++) {
                        const float a = x[s][t], b = x[s | st][t];
                        x[s][t] = c * a + sn * b;
                        x[s | st][t] = sn * a - c * b;
                    }
                }
#pragma unroll
                for (int t = 0; t < G; t++) {
                    if ((t & st) || !cv[t | st]) continue;
                    const float c = sfv[it][l][t], sn = sfv[it][l][t | st];
#pragma unroll
                    for (int s = 0; s < G; s++) {
                        const float a = x[s][t], b = x[s][t | st];
                        x[s][t] = c * a + sn * b;
                        x[s][t | st] = sn * a - c * b;
                    }
                }
                continue;
            }
#pragma unroll
            for (int s = 0; s < G; s++) {
                if ((s & st) || !rv[s | st]) continue;
#pragma unroll
                for (int t = 0; t < G; t++) {
                    float a = x[s][t], b = x[s | st][t];
                    x[s][t] = a + b;
                    x[s | st][t] = a - b;
                }
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                if ((t & st) || !cv[t | st]) continue;
#pragma unroll
                for (int s = 0; s < G; s++) {
                    float a = x[s][t], b = x[s][t | st];
                    x[s][t] = a + b;
                    x[s][t | st] = a - b;
                }
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                const float fv = sfv[it][l][t];
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] = (x[s][t] * fu[l][s]) * fv;
            }
        }
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++)
                if (rv[s] && cv[t]) __stcs(Aout + row[s] + col[t] * lda_out, x[s][t]);
    }
}

static rbt_status transform2_f32math(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                                     const double *Ain, int64_t lda_in, float *Aout, int64_t lda_out,
                                     cudaStream_t stream, int64_t align = 1, bool rot = false)
{
    const int ds = eff_depth(n, d);
    if (ds == 0 || ds > 3)
        return transform2<float>(n, d, U, V, ldw, Ain, lda_in, Aout, lda_out, 3, stream, align, rot);
    ProfScope ps(kProfTransform, stream);
    const int64_t m = ref_size(n, d, align);
    const int64_t h = m >> ds;
    // two column groups per thread: the row coefficients are shared by both,
    // and each thread keeps 2^(2 ds) double loads of one group in flight at a
    // time (four groups per thread measured 40% slower on this access pattern)
    const int gpt = kF32Gpt;
    dim3 grid((unsigned)cdiv(h, kTX), (unsigned)cdiv(h, gpt));
    const int pre_lo = ds + 1, pre_hi = d;
#define RBT_F32_LAUNCH(LL, RR) \
    fused2_f32_kernel<LL, RR><<<grid, kTX, 0, stream>>>(n, h, h, ds, pre_lo, pre_hi, U, V, ldw, Ain, lda_in, Aout, lda_out, gpt)
    switch (ds * 2 + (rot ? 1 : 0)) {
    case 2: RBT_F32_LAUNCH(1, false); break;
    case 3: RBT_F32_LAUNCH(1, true); break;
    case 4: RBT_F32_LAUNCH(2, false); break;
    case 5: RBT_F32_LAUNCH(2, true); break;
    case 6: RBT_F32_LAUNCH(3, false); break;
    default: RBT_F32_LAUNCH(3, true); break;
    }
#undef RBT_F32_LAUNCH
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

// ------------------------------------ double-float working copy, FP32 math

// double -> float pair (hi + lo with |lo| <= ulp(hi) / 2, within 2^-48 |x|)
// by integer operations on the bit pattern, for exponents whose hi and lo
// land in the float normal range; the rest (zero, subnormals, very large or
// small magnitudes, inf, nan) through the conversion unit.
__device__ __forceinline__ df64 split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 949 || e > 1149) {
        const float hi = __double2float_rn(x);
        return df64(hi, __double2float_rn(x - (double)hi));
    }
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned long long hm = (M + 0x0FFFFFFFull + ((M >> 29) & 1ull)) >> 29;  // 24 bits, or 2^24
    const long long rem = (long long)M - (long long)(hm << 29);                     // |rem| <= 2^28
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __int_as_float((int)((((unsigned)(e - 896) << 23) + (unsigned)(hm - (1ull << 23))) | sign));
    float lo = (float)(int)rem * __int_as_float((e - 1075 + 127) << 23);
    return df64(hi, sign ? -lo : lo);
}

// The double-float working copy: the same single pass as the float one, with
// every layer in double-float arithmetic on the FP32 pipes (about 2^-44
// relative to |U|^T |A| |V| per entry; the refinement measures against A in
// double).  HBM-bound (16 bytes per entry) where the double-arithmetic pass
// is FP64-ALU bound.
template <int L, bool ROT = false>
__global__ void __launch_bounds__(kTX)
fused2_df64math_kernel(int64_t n, int64_t h, int64_t ngroups, int k_hi, int pre_lo, int pre_hi,
                       const double *__restrict__ U, const double *__restrict__ V, int64_t ldw,
                       const double *__restrict__ Ain, int64_t lda_in, df64 *__restrict__ Aout, int64_t lda_out,
                       int gpt)
{
    constexpr int G = 1 << L;
    constexpr double kSd = 0.70710678118654752440;
    constexpr float kSh = (float)kSd;
    constexpr float kSl = (float)(kSd - (double)kSh);
    const df64 kS(kSh, kSl);
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
    df64 fu[L][G], pu[G];
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int k = k_hi - l;
        const int st = 1 << l;
#pragma unroll
        for (int s = 0; s < G; s++) {
            const df64 u = rv[s] ? split_double(__ldg(U + row[s] + (int64_t)(k - 1) * ldw)) : df64(0);
            fu[l][s] = (!ROT && rv[s | st]) ? u * kS : u;
        }
    }
#pragma unroll
    for (int s = 0; s < G; s++) {
        df64 p(1.f);
        for (int k = pre_lo; k <= pre_hi; k++)
            p = p * (rv[s] ? split_double(__ldg(U + row[s] + (int64_t)(k - 1) * ldw)) : df64(0));
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
        double a[G][G];
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++) a[s][t] = (rv[s] && cv[t]) ? __ldcs(Ain + row[s] + col[t] * lda_in) : 0.0;
        df64 x[G][G];
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++) x[s][t] = split_double(a[s][t]);
        if (has_pre) {
#pragma unroll
            for (int t = 0; t < G; t++) {
                df64 p(1.f);
                for (int k = pre_lo; k <= pre_hi; k++)
                    p = p * (cv[t] ? split_double(__ldg(V + col[t] + (int64_t)(k - 1) * ldw)) : df64(0));
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] = x[s][t] * (pu[s] * p);
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
                    const df64 c = fu[l][s], sn = fu[l][s | st];
#pragma unroll
                    for (int t = 0; t < G; t++) {
                        const df64 p = x[s][t], q = x[s | st][t];
                        x[s][t] = c * p + sn * q;
                        x[s | st][t] = sn * p - c * q;
                    }
                }
                df64 fv[G];
#pragma unroll
                for (int t = 0; t < G; t++)
                    fv[t] = cv[t] ? split_double(__ldg(V + col[t] + (int64_t)(k - 1) * ldw)) : df64(0);
#pragma unroll
                for (int t = 0; t < G; t++) {
                    if ((t & st) || !cv[t | st]) continue;
                    const df64 c = fv[t], sn = fv[t | st];
#pragma unroll
                    for (int s = 0; s < G; s++) {
                        const df64 p = x[s][t], q = x[s][t | st];
                        x[s][t] = c * p + sn * q;
                        x[s][t | st] = sn * p - c * q;
                    }
                }
                continue;
            }
#pragma unroll
            for (int s = 0; s < G; s++) {
                if ((s & st) || !rv[s | st]) continue;
#pragma unroll
                for (int t = 0; t < G; t++) {
                    const df64 p = x[s][t], q = x[s | st][t];
                    x[s][t] = p + q;
                    x[s | st][t] = p - q;
                }
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                if ((t & st) || !cv[t | st]) continue;
#pragma unroll
                for (int s = 0; s < G; s++) {
                    const df64 p = x[s][t], q = x[s][t | st];
                    x[s][t] = p + q;
                    x[s][t | st] = p - q;
                }
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                const df64 v = cv[t] ? split_double(__ldg(V + col[t] + (int64_t)(k - 1) * ldw)) : df64(0);
                const df64 fv = cv[t | st] ? v * kS : v;
#pragma unroll
                for (int s = 0; s < G; s++) x[s][t] = (x[s][t] * fu[l][s]) * fv;
            }
        }
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++)
                if (rv[s] && cv[t])
                    __stcs(reinterpret_cast<float2 *>(Aout + row[s] + col[t] * lda_out), make_float2(x[s][t].hi, x[s][t].lo));
    }
}

static rbt_status transform2_df64math(int64_t n, int d, const double *U, const double *V, int64_t ldw,
                                      const double *Ain, int64_t lda_in, df64 *Aout, int64_t lda_out,
                                      cudaStream_t stream, int64_t align = 1, bool rot = false)
{
    const int ds = eff_depth(n, d);
    if (ds == 0 || ds > 3)
        return transform2<df64>(n, d, U, V, ldw, Ain, lda_in, Aout, lda_out, 3, stream, align, rot);
    ProfScope ps(kProfTransform, stream);
    const int64_t m = ref_size(n, d, align);
    const int64_t h = m >> ds;
    const int gpt = 2;
    dim3 grid((unsigned)cdiv(h, kTX), (unsigned)cdiv(h, gpt));
    const int pre_lo = ds + 1, pre_hi = d;
#define RBT_DF_LAUNCH(LL, RR) \
    fused2_df64math_kernel<LL, RR><<<grid, kTX, 0, stream>>>(n, h, h, ds, pre_lo, pre_hi, U, V, ldw, Ain, lda_in, Aout, lda_out, gpt)
    switch (ds * 2 + (rot ? 1 : 0)) {
    case 2: RBT_DF_LAUNCH(1, false); break;
    case 3: RBT_DF_LAUNCH(1, true); break;
    case 4: RBT_DF_LAUNCH(2, false); break;
    case 5: RBT_DF_LAUNCH(2, true); break;
    case 6: RBT_DF_LAUNCH(3, false); break;
    default: RBT_DF_LAUNCH(3, true); break;
    }
#undef RBT_DF_LAUNCH
    RBT_LAUNCH_CHECK();
    return RBT_OK;
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
    if (n < 0 || d < 0 || d > 62 || align < 0 || prec < RBT_F64 || prec > RBT_DF64TC) return RBT_ERR_ARG;
    if (kind != RBT_KIND_SCALED && kind != RBT_KIND_ROTATION) return RBT_ERR_ARG;
    const bool rot = kind == RBT_KIND_ROTATION;
    int64_t mn = n > 1 ? n : 1;
    if (lda_in < mn || lda_out < mn || (d > 0 && ldw < mn)) return RBT_ERR_ARG;
    if (n == 0) return RBT_OK;
    if (!A_in || !A_out || (d > 0 && (!U || !V))) return RBT_ERR_ARG;
    size_t es = prec == RBT_F64 || prec == RBT_DF64 || prec == RBT_DF64TC ? 8 : 4;
    if ((const void *)A_in == A_out || overlap_bad(A_in, lda_in, A_out, lda_out, n, 8, es)) return RBT_ERR_ARG;
    if (prec == RBT_F64)
        return apply_2sided_f64(n, d, align, rot, U, V, ldw, A_in, lda_in, (double *)A_out, lda_out, stream);
    if (eff_depth(n, d) > 3) return RBT_ERR_UNSUPPORTED;  // one pass must cover every layer
    if (prec == RBT_DF64 || prec == RBT_DF64TC)
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
