// Device building blocks of the butterfly transforms, shared by the
// whole-matrix kernels (rbt_transform.cu) and the batched solver (batched.cu).
//
// Index structure (Eq. rbt-depth-d with the alignment rule): with reference
// size m and half sizes h_k = m / 2^k, layer k pairs row i with i + h_k.  For
// a run of layers k_lo..k_hi (L = k_hi - k_lo + 1) each row is
// i = (c 2^L + s) h + r with h = h_{k_hi}; layer k pairs local index s with
// s + 2^(k_hi - k), so the 2^L rows of a group (c, r) are closed under those
// layers.  A pair exists when its bottom row is < n; otherwise the top row is
// a nu row of Eq. (O-matrix-definition) and passes through unscaled.
#pragma once

#include "common.cuh"
#include "df64.cuh"

namespace rbt {

constexpr double kInvSqrt2d = 0.70710678118654752440084436210485;

// Counter-based SplitMix64 keyed by (seed, side, layer, row): a uniform u on
// [0, 1) with 53 random bits.
__device__ __forceinline__ double counter_u(uint64_t seed, int side, int layer, int64_t i)
{
    uint64_t z = (seed ^ ((uint64_t)side << 62) ^ ((uint64_t)layer << 48) ^ (uint64_t)i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53;
}

// Sec. 6: exp(r/20), r uniform on [-1, 1).
__device__ __forceinline__ double coef_value(uint64_t seed, int side, int layer, int64_t i)
{
    return exp((2.0 * counter_u(seed, side, layer, i) - 1.0) / 20.0);
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Rotation form of the butterflies (Sec. 3, the block-rotation variant):
// each pair (top i, bottom i + h_k) of layer k turns by the angle 2 pi u,
// u from the counter of its top row; the packed column k-1 holds cos at the
// top row, sin at the bottom row, and 1 at nu rows and in layers k > d_s
// (the identity of a rotation by 0).
__device__ __forceinline__ double rot_value(uint64_t seed, int side, int layer, int64_t i, int64_t n, int64_t m,
                                            int ds)
{
    if (layer > ds) return 1.0;
    const int64_t h = m >> layer;
    const bool top = (i % (2 * h)) < h;
    if (top && i + h >= n) return 1.0;
    const double th = kTwoPi * counter_u(seed, side, layer, top ? i : i - h);
    return top ? cos(th) : sin(th);
}

template <typename T> __device__ __forceinline__ T narrow_to(double v);
template <> __device__ __forceinline__ double narrow_to<double>(double v) { return v; }
template <> __device__ __forceinline__ float narrow_to<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ df64 narrow_to<df64>(double v) { return df_from_double(v); }

// Two-sided transform of one (row group, column group) pair over layers
// k_hi .. k_hi - L + 1, preceded by the diagonal-only layers pre_lo..pre_hi.
template <int L, typename TO>
__device__ __forceinline__ void transform_group(int64_t n, int64_t h, int k_hi, int pre_lo, int pre_hi,
                                                const double *__restrict__ U, const double *__restrict__ V,
                                                int64_t ldw, const double *Ain, int64_t lda_in, TO *Aout,
                                                int64_t lda_out, int64_t gr, int64_t gc)
{
    constexpr int G = 1 << L;
    const int64_t cr = gr / h, rr = gr - cr * h;
    const int64_t cc = gc / h, rc = gc - cc * h;
    int64_t row[G], col[G];
    bool rv[G], cv[G];
#pragma unroll
    for (int s = 0; s < G; s++) {
        row[s] = (cr * G + s) * h + rr;
        rv[s] = row[s] < n;
        col[s] = (cc * G + s) * h + rc;
        cv[s] = col[s] < n;
    }
    double x[G][G];
#pragma unroll
    for (int t = 0; t < G; t++)
#pragma unroll
        for (int s = 0; s < G; s++) x[s][t] = (rv[s] && cv[t]) ? Ain[row[s] + col[t] * lda_in] : 0.0;
    if (pre_hi >= pre_lo) {
#pragma unroll
        for (int s = 0; s < G; s++) {
            double pu = 1.0, pv = 1.0;
            for (int k = pre_lo; k <= pre_hi; k++) {
                pu *= rv[s] ? U[row[s] + (int64_t)(k - 1) * ldw] : 0.0;
                pv *= cv[s] ? V[col[s] + (int64_t)(k - 1) * ldw] : 0.0;
            }
#pragma unroll
            for (int t = 0; t < G; t++) {
                x[s][t] *= pu;
                x[t][s] *= pv;
            }
        }
    }
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int k = k_hi - l;
        const int st = 1 << l;
#pragma unroll
        for (int s = 0; s < G; s++) {
            if ((s & st) || !rv[s | st]) continue;
#pragma unroll
            for (int t = 0; t < G; t++) {
                double a = x[s][t], b = x[s | st][t];
                x[s][t] = a + b;
                x[s | st][t] = a - b;
            }
        }
#pragma unroll
        for (int t = 0; t < G; t++) {
            if ((t & st) || !cv[t | st]) continue;
#pragma unroll
            for (int s = 0; s < G; s++) {
                double a = x[s][t], b = x[s][t | st];
                x[s][t] = a + b;
                x[s][t | st] = a - b;
            }
        }
        double fu[G], fv[G];
#pragma unroll
        for (int s = 0; s < G; s++) {
            double u = rv[s] ? U[row[s] + (int64_t)(k - 1) * ldw] : 0.0;
            double v = cv[s] ? V[col[s] + (int64_t)(k - 1) * ldw] : 0.0;
            fu[s] = rv[s | st] ? u * kInvSqrt2d : u;
            fv[s] = cv[s | st] ? v * kInvSqrt2d : v;
        }
#pragma unroll
        for (int t = 0; t < G; t++)
#pragma unroll
            for (int s = 0; s < G; s++) x[s][t] = (x[s][t] * fu[s]) * fv[t];
    }
#pragma unroll
    for (int t = 0; t < G; t++)
#pragma unroll
        for (int s = 0; s < G; s++)
            if (rv[s] && cv[t]) Aout[row[s] + col[t] * lda_out] = narrow_to<TO>(x[s][t]);
}

// transform_group by 2^L cooperating lanes (consecutive lanes of one warp,
// mask = their bits): lane s of the group holds row s of the 2^L x 2^L block,
// the column butterflies stay inside the lane and the row butterflies pair
// lanes by shuffles.  Every entry takes the same operations in the same
// order as in transform_group, so the results are bit for bit the same; a
// lane holds 2^L values instead of 4^L (the depth-3 group is 64 doubles).
template <int L, typename TO>
__device__ __forceinline__ void transform_group_rows(int64_t n, int64_t h, int k_hi, int pre_lo, int pre_hi,
                                                     const double *__restrict__ U, const double *__restrict__ V,
                                                     int64_t ldw, const double *Ain, int64_t lda_in, TO *Aout,
                                                     int64_t lda_out, int64_t gr, int64_t gc, int s, unsigned mask)
{
    constexpr int G = 1 << L;
    const int64_t cr = gr / h, rr = gr - cr * h;
    const int64_t cc = gc / h, rc = gc - cc * h;
    auto row_of = [&](int q) { return (cr * G + q) * h + rr; };
    const int64_t row = row_of(s);
    const bool rv = row < n;
    int64_t col[G];
    bool cv[G];
#pragma unroll
    for (int t = 0; t < G; t++) {
        col[t] = (cc * G + t) * h + rc;
        cv[t] = col[t] < n;
    }
    double x[G];
#pragma unroll
    for (int t = 0; t < G; t++) x[t] = (rv && cv[t]) ? Ain[row + col[t] * lda_in] : 0.0;
    if (pre_hi >= pre_lo) {
        // entry (s, t) takes its row factor first when s <= t, its column factor first otherwise
        double pu = 1.0;
        for (int k = pre_lo; k <= pre_hi; k++) pu *= rv ? U[row + (int64_t)(k - 1) * ldw] : 0.0;
#pragma unroll
        for (int t = 0; t < G; t++) {
            double pv = 1.0;
            for (int k = pre_lo; k <= pre_hi; k++) pv *= cv[t] ? V[col[t] + (int64_t)(k - 1) * ldw] : 0.0;
            x[t] = s <= t ? (x[t] * pu) * pv : (x[t] * pv) * pu;
        }
    }
#pragma unroll
    for (int l = 0; l < L; l++) {
        const int k = k_hi - l;
        const int st = 1 << l;
        const bool top = !(s & st);
        const bool pair = row_of(s | st) < n;  // the pair's bottom row exists
#pragma unroll
        for (int t = 0; t < G; t++) {
            const double o = __shfl_xor_sync(mask, x[t], st, G);
            if (pair) x[t] = top ? x[t] + o : o - x[t];
        }
#pragma unroll
        for (int t = 0; t < G; t++) {
            if ((t & st) || !cv[t | st]) continue;
            const double a = x[t], b = x[t | st];
            x[t] = a + b;
            x[t | st] = a - b;
        }
        const double u = rv ? U[row + (int64_t)(k - 1) * ldw] : 0.0;
        const double fu = pair ? u * kInvSqrt2d : u;
#pragma unroll
        for (int t = 0; t < G; t++) {
            const double v = cv[t] ? V[col[t] + (int64_t)(k - 1) * ldw] : 0.0;
            const double fv = cv[t | st] ? v * kInvSqrt2d : v;
            x[t] = (x[t] * fu) * fv;
        }
    }
#pragma unroll
    for (int t = 0; t < G; t++)
        if (rv && cv[t]) Aout[row + col[t] * lda_out] = narrow_to<TO>(x[t]);
}

// One-sided transform of one row group of one column B (in place):
// trans = 1: B <- W^T B (layers k_hi..k_lo, each B_k then R_k; diagonal-only
// layers ext_lo..ext_hi first); trans = 0: B <- W B (layers k_lo..k_hi, each
// R_k then B_k; diagonal-only layers last).
//
// ROT: the rotation form instead (R_k = I): each pair (a, b) with packed
// (c, s) becomes (c a + s b, s a - c b); B_k is symmetric, so W^T applies
// the same layers in the reverse order.
template <int L, bool ROT = false>
__device__ __forceinline__ void vec_group(int64_t n, int64_t h, int k_hi, int trans, int ext_lo, int ext_hi,
                                          const double *__restrict__ W, int64_t ldw, double *B, int64_t gr)
{
    constexpr int G = 1 << L;
    const int64_t cr = gr / h, rr = gr - cr * h;
    int64_t row[G];
    bool rv[G];
    double x[G], ext[G];
#pragma unroll
    for (int s = 0; s < G; s++) {
        row[s] = (cr * G + s) * h + rr;
        rv[s] = row[s] < n;
        x[s] = rv[s] ? B[row[s]] : 0.0;
        double p = 1.0;
        for (int k = ext_lo; k <= ext_hi; k++) p *= rv[s] ? W[row[s] + (int64_t)(k - 1) * ldw] : 0.0;
        ext[s] = p;
    }
    if (trans && ext_hi >= ext_lo) {
#pragma unroll
        for (int s = 0; s < G; s++) x[s] *= ext[s];
    }
#pragma unroll
    for (int li = 0; li < L; li++) {
        const int l = trans ? li : (L - 1 - li);
        const int k = k_hi - l;
        const int st = 1 << l;
        if (ROT) {
#pragma unroll
            for (int s = 0; s < G; s++) {
                if ((s & st) || !rv[s | st]) continue;
                const double c = W[row[s] + (int64_t)(k - 1) * ldw], sn = W[row[s | st] + (int64_t)(k - 1) * ldw];
                const double a = x[s], b = x[s | st];
                x[s] = c * a + sn * b;
                x[s | st] = sn * a - c * b;
            }
            continue;
        }
        if (!trans) {
#pragma unroll
            for (int s = 0; s < G; s++) x[s] *= rv[s] ? W[row[s] + (int64_t)(k - 1) * ldw] : 0.0;
        }
#pragma unroll
        for (int s = 0; s < G; s++) {
            if ((s & st) || !rv[s | st]) continue;
            double a = x[s], b = x[s | st];
            x[s] = (a + b) * kInvSqrt2d;
            x[s | st] = (a - b) * kInvSqrt2d;
        }
        if (trans) {
#pragma unroll
            for (int s = 0; s < G; s++) x[s] *= rv[s] ? W[row[s] + (int64_t)(k - 1) * ldw] : 0.0;
        }
    }
    if (!trans && ext_hi >= ext_lo) {
#pragma unroll
        for (int s = 0; s < G; s++) x[s] *= ext[s];
    }
#pragma unroll
    for (int s = 0; s < G; s++)
        if (rv[s]) B[row[s]] = x[s];
}

}  // namespace rbt
