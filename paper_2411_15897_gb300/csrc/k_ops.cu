// Matrix-free kernels of the outer system and the preconditioner's two
// coupling steps:
//   * y = H x (or y = b - H x) in FP64, Eq. 2.6;
//   * t_p = B r_u - A_p r_p, the distributed right-hand side (Eq. 3.1-3.3);
//   * s_u = r_u - B^T e_p, the back-substitution of the block-triangular
//     solve with P = [A B^T; 0 H_p] (Eq. 3.5).
#include "bah_internal.cuh"
#include "df.cuh"
#include "op_rows.cuh"

namespace bah {

template <class V>
__device__ __forceinline__ double2 ld64(const V* p, int idx) {
    V v = p[idx];
    return make_double2((double)v.x, (double)v.y);
}
__device__ __forceinline__ double2 ld64(const float4* p, int idx) { return cdf_to_double2(p[idx]); }
// preconditioner input in the preconditioner's real type R
template <class R> __device__ __forceinline__ R ldr_in(const double2& v, int c) { return (R)(c ? v.y : v.x); }
__device__ __forceinline__ float ldf_in(const double2& v, bool im) { return (float)(im ? v.y : v.x); }
template <class R> struct InLoad;
template <> struct InLoad<double> {
    __device__ static double2 get(const double2* p, size_t i) { return p[i]; }
    __device__ static double2 get(const float4* p, size_t i) { return cdf_to_double2(p[i]); }
};
template <> struct InLoad<float> {
    __device__ static float2 get(const double2* p, size_t i) { const double2 v = p[i]; return make_float2((float)v.x, (float)v.y); }
    __device__ static float2 get(const float4* p, size_t i) { const float4 v = p[i]; return make_float2(v.x + v.y, v.z + v.w); }
};
__device__ __forceinline__ void st_out(double2* y, size_t i, double2 v) { y[i] = v; }
__device__ __forceinline__ void st_out(float4* y, size_t i, double2 v) { y[i] = cdf_from_double2(v); }

// ---------------------------------------------------------------------------
// y = H x  (b == nullptr)  or  y = b - H x,  one cell per thread.
// conj != 0 applies H^H = conj(H) (H is complex symmetric).
// ---------------------------------------------------------------------------
template <class Vin, class Vout>
__global__ void __launch_bounds__(256) k_elastic_apply(OpCoef c, const Vin* __restrict__ x, Vout* __restrict__ y,
                                                       const double2* __restrict__ b, int conj, RhsStride rs) {
    pdl_prologue();
    const int n1 = c.n1, n2 = c.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.y;
    if (t >= np || (rs.active && !rs.active[rr])) return;
    x += rr * rs.s0;
    y += rr * rs.s1;
    if (b) b += rr * rs.s2;
    const int i = t % n1, j = t / n1;
    const Vin* x1 = x;
    const Vin* x2 = x + np;
    const Vin* xp = x + 2 * np;
    const double2 z = make_double2(0.0, 0.0);
    auto U1 = [&](int ii, int jj) { return (ii >= 1 && ii < n1 && jj >= 0 && jj < n2) ? ld64(x1, jj * n1 + ii) : z; };
    auto U2 = [&](int ii, int jj) { return (ii >= 0 && ii < n1 && jj >= 1 && jj < n2) ? ld64(x2, jj * n1 + ii) : z; };
    auto P = [&](int g) { return ld64(xp, g); };
    double2 y1, y2, yp;
    elastic_rows(c, i, j, t, conj ? -1.0 : 1.0, U1, U2, P, y1, y2, yp);
    if (b) {
        if (i >= 1) y1 = csub(b[t], y1);
        if (j >= 1) y2 = csub(b[np + t], y2);
        yp = csub(b[2 * np + t], yp);
    }
    st_out(y, t, y1);
    st_out(y, np + t, y2);
    st_out(y, 2 * np + t, yp);
}

// ---------------------------------------------------------------------------
// y = H x for an FP32 x (the flexible basis in mixed mode), in double-float
// arithmetic: every coefficient is a double-float pair, every product an
// error-free FP32 product (FMA) and every sum a two-sum, so the result matches
// the FP64 kernel to about 2^-47 relative without FP64 instructions.  Same
// stencil as k_elastic_apply (Eq. 2.6), y = H x only.
// ---------------------------------------------------------------------------
// the double-float result (hi, lo per real) as a double-float pair, or rounded
// once to FP64 (hi + lo is exact in FP64: both parts are FP32 values of one
// 48-bit significand)
__device__ __forceinline__ void st_dfa(float4* y, size_t i, const float4& v) { y[i] = v; }
__device__ __forceinline__ void st_dfa(double2* y, size_t i, const float4& v) {
    y[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
template <class Vout>
__global__ void __launch_bounds__(256) k_elastic_apply_dfa(OpCoefDF c, const float2* __restrict__ x,
                                                           Vout* __restrict__ y, RhsStride rs) {
    pdl_prologue();
    const int n1 = c.n1, n2 = c.n2, np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.y;
    if (t >= np || (rs.active && !rs.active[rr])) return;
    x += rr * rs.s0;
    y += rr * rs.s1;
    const int i = t % n1, j = t / n1;
    const float2* x1 = x;
    const float2* x2 = x + np;
    const float2* xp = x + 2 * np;
    const float2 z = make_float2(0.f, 0.f);
    auto U1 = [&](int ii, int jj) { return (ii >= 1 && ii < n1 && jj >= 0 && jj < n2) ? x1[jj * n1 + ii] : z; };
    auto U2 = [&](int ii, int jj) { return (ii >= 0 && ii < n1 && jj >= 1 && jj < n2) ? x2[jj * n1 + ii] : z; };
    const float2 p = xp[t];
    const dfl ihx = df_of(c.ihx), ihz = df_of(c.ihz);
    const dfl zero = {0.f, 0.f};
    // acc -= k v (k real double-float, v complex float)
    auto sub_kv = [&](dfacc& ar, dfacc& ai, dfl k, float2 v) {
        ar.add(df_neg(df_mul_f(k, v.x)));
        ai.add(df_neg(df_mul_f(k, v.y)));
    };
    float4 y1 = make_float4(0.f, 0.f, 0.f, 0.f), y2 = y1;
    if (i >= 1) {
        // u1 row: (diagonal) u - neighbours + (grad_h p)_1
        const float2 u = U1(i, j);
        const float4 d = c.d1[t];
        const dfl dr = re_of(d), di = im_of(d);
        dfacc ar, ai;
        ar.add(df_mul_f(dr, u.x));
        ar.add(df_neg(df_mul_f(di, u.y)));
        ai.add(df_mul_f(dr, u.y));
        ai.add(df_mul_f(di, u.x));
        sub_kv(ar, ai, df_of(c.cx[t - 1]), U1(i - 1, j));
        sub_kv(ar, ai, df_of(c.cx[t]), U1(i + 1, j));
        sub_kv(ar, ai, df_of(c.nz[t]), U1(i, j - 1));
        sub_kv(ar, ai, (j + 1 < n2) ? df_of(c.nz[t + n1]) : zero, U1(i, j + 1));
        const float2 pw = xp[t - 1];
        ar.add(df_mul(ihx, df_diff_f(p.x, pw.x)));
        ai.add(df_mul(ihx, df_diff_f(p.y, pw.y)));
        y1 = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
    }
    if (j >= 1) {
        const float2 u = U2(i, j);
        const float4 d = c.d2[t];
        const dfl dr = re_of(d), di = im_of(d);
        dfacc ar, ai;
        ar.add(df_mul_f(dr, u.x));
        ar.add(df_neg(df_mul_f(di, u.y)));
        ai.add(df_mul_f(dr, u.y));
        ai.add(df_mul_f(di, u.x));
        sub_kv(ar, ai, df_of(c.cz[t - n1]), U2(i, j - 1));
        sub_kv(ar, ai, df_of(c.cz[t]), U2(i, j + 1));
        sub_kv(ar, ai, df_of(c.nx[t]), U2(i - 1, j));
        sub_kv(ar, ai, (i + 1 < n1) ? df_of(c.nx[t + 1]) : zero, U2(i + 1, j));
        const float2 ps = xp[t - n1];
        ar.add(df_mul(ihz, df_diff_f(p.x, ps.x)));
        ai.add(df_mul(ihz, df_diff_f(p.y, ps.y)));
        y2 = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
    }
    // p row: B u - C p
    const float2 u1c = U1(i, j), u1e = U1(i + 1, j), u2c = U2(i, j), u2n = U2(i, j + 1);
    const dfl ci = df_of(c.cinv[t]);
    dfacc pr, pi;
    pr.add(df_mul(ihx, df_diff_f(u1c.x, u1e.x)));
    pr.add(df_mul(ihz, df_diff_f(u2c.x, u2n.x)));
    pr.add(df_neg(df_mul_f(ci, p.x)));
    pi.add(df_mul(ihx, df_diff_f(u1c.y, u1e.y)));
    pi.add(df_mul(ihz, df_diff_f(u2c.y, u2n.y)));
    pi.add(df_neg(df_mul_f(ci, p.y)));
    st_dfa(y, t, y1);
    st_dfa(y, np + t, y2);
    st_dfa(y, 2 * np + t, make_float4(pr.hi, pr.lo, pi.hi, pi.lo));
}
void launch_elastic_apply_dfa(const OpCoefDF& c, const float2* x, float4* y, cudaStream_t st, int nrhs, RhsStride rs) {
    const int np = c.n1 * c.n2;
    launch_pdl(k_elastic_apply_dfa<float4>, dim3(dim3((np + 255) / 256, nrhs)), dim3(256), 0, st, c, x, y, rs);
}
void launch_elastic_apply_dfa(const OpCoefDF& c, const float2* x, double2* y, cudaStream_t st, int nrhs, RhsStride rs) {
    const int np = c.n1 * c.n2;
    launch_pdl(k_elastic_apply_dfa<double2>, dim3(dim3((np + 255) / 256, nrhs)), dim3(256), 0, st, c, x, y, rs);
}
__global__ void k_to_df(const double* __restrict__ s, float2* __restrict__ d, size_t n) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e < n) {
        const dfl v = df_from_double(s[e]);
        d[e] = make_float2(v.hi, v.lo);
    }
}
__global__ void k_to_df_c(const double2* __restrict__ s, float4* __restrict__ d, size_t n) {
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (e < n) d[e] = cdf_from_double2(s[e]);
}
void launch_to_df(const double* src, float2* dst, size_t n, cudaStream_t st) {
    k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
}
void launch_to_df_c(const double2* src, float4* dst, size_t n, cudaStream_t st) {
    k_to_df_c<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
}

template <class Vin>
void launch_elastic_apply(const OpCoef& c, const Vin* x, double2* y, const double2* b, int conj, cudaStream_t st,
                          int nrhs, RhsStride rs) {
    int np = c.n1 * c.n2;
    launch_pdl(k_elastic_apply<Vin, double2>, dim3(dim3((np + 255) / 256, nrhs)), dim3(256), 0, st, c, x, y, b, conj, rs);
}
template <class Vin>
void launch_elastic_apply_df(const OpCoef& c, const Vin* x, float4* y, cudaStream_t st, int nrhs, RhsStride rs) {
    int np = c.n1 * c.n2;
    launch_pdl(k_elastic_apply<Vin, float4>, dim3(dim3((np + 255) / 256, nrhs)), dim3(256), 0, st, c, x, y, nullptr, 0, rs);
}
template void launch_elastic_apply_df<double2>(const OpCoef&, const double2*, float4*, cudaStream_t, int, RhsStride);
template void launch_elastic_apply_df<float2>(const OpCoef&, const float2*, float4*, cudaStream_t, int, RhsStride);
template void launch_elastic_apply<double2>(const OpCoef&, const double2*, double2*, const double2*, int, cudaStream_t,
                                            int, RhsStride);
template void launch_elastic_apply<float2>(const OpCoef&, const float2*, double2*, const double2*, int, cudaStream_t,
                                           int, RhsStride);

// ---------------------------------------------------------------------------
// t_p = B r_u - A_p r_p   (r in FP64, t_p in the preconditioner's precision)
// ---------------------------------------------------------------------------
template <int MODE, class RIN>
__global__ void __launch_bounds__(256) k_distributor(int n1, int n2, typename Prec<MODE>::R ihx,
                                                     typename Prec<MODE>::R ihz,
                                                     Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC> f,
                                                     const RIN* __restrict__ r, typename Prec<MODE>::V* __restrict__ tp,
                                                     RhsStride rs) {
    pdl_prologue();
    using V = typename Prec<MODE>::V;
    using R = typename Prec<MODE>::R;
    const int np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.y;
    if (t >= np || (rs.active && !rs.active[rr])) return;
    r += rr * rs.s0;
    tp += rr * rs.s1;
    const int i = t % n1, j = t / n1;
    auto L = [&](int idx) { return InLoad<R>::get(r, idx); };
    const V z = czero<V>();
    const V u1c = (i >= 1) ? L(t) : z;
    const V u1e = (i + 1 < n1) ? L(t + 1) : z;
    const V u2c = (j >= 1) ? L(np + t) : z;
    const V u2n = (j + 1 < n2) ? L(np + t + n1) : z;
    // B r_u
    V acc = cmk<V>(ihx * (u1c.x - u1e.x) + ihz * (u2c.x - u2n.x), ihx * (u1c.y - u1e.y) + ihz * (u2c.y - u2n.y));
    // - A_p r_p,  A_p = B B^T diag(mu) - omega^2 diag(rho~): off-diagonal (c, n) = -mu_n / h^2
    const V pc = L(2 * np + t);
    V ap = cmul(ldc(f.dAp[t]), pc);
    if (i >= 1) { R k = ldr(f.cx[t - 1]); V q = L(2 * np + t - 1); ap.x -= k * q.x; ap.y -= k * q.y; }
    if (i + 1 < n1) { R k = ldr(f.cx[t + 1]); V q = L(2 * np + t + 1); ap.x -= k * q.x; ap.y -= k * q.y; }
    if (j >= 1) { R k = ldr(f.cz[t - n1]); V q = L(2 * np + t - n1); ap.x -= k * q.x; ap.y -= k * q.y; }
    if (j + 1 < n2) { R k = ldr(f.cz[t + n1]); V q = L(2 * np + t + n1); ap.x -= k * q.x; ap.y -= k * q.y; }
    tp[t] = csub(acc, ap);
}

template <int MODE, class RIN>
void launch_distributor(int n1, int n2, double ihx, double ihz,
                        const Fine5<typename Prec<MODE>::C, typename Prec<MODE>::CC>& f5, const RIN* r,
                        typename Prec<MODE>::V* tp, cudaStream_t st, int nrhs, RhsStride rs) {
    int np = n1 * n2;
    launch_pdl(k_distributor<MODE, RIN>, dim3(dim3((np + 255) / 256, nrhs)), dim3(256), 0, st, n1, n2, (typename Prec<MODE>::R)ihx,
                                                                       (typename Prec<MODE>::R)ihz, f5, r, tp, rs);
}
template void launch_distributor<BAH_FP64, double2>(int, int, double, double, const Fine5<double, double2>&,
                                                    const double2*, double2*, cudaStream_t, int, RhsStride);
template void launch_distributor<BAH_MIXED, double2>(int, int, double, double,
                                                     const Fine5<__nv_bfloat16, __nv_bfloat162>&, const double2*,
                                                     float2*, cudaStream_t, int, RhsStride);
template void launch_distributor<BAH_FP64, float4>(int, int, double, double, const Fine5<double, double2>&,
                                                   const float4*, double2*, cudaStream_t, int, RhsStride);
template void launch_distributor<BAH_MIXED, float4>(int, int, double, double,
                                                    const Fine5<__nv_bfloat16, __nv_bfloat162>&, const float4*,
                                                    float2*, cudaStream_t, int, RhsStride);

// ---------------------------------------------------------------------------
// s_u = r_u - B^T e_p  (B^T = grad_h onto the interior faces)
// ---------------------------------------------------------------------------
template <int MODE, class RIN>
__global__ void __launch_bounds__(256) k_u_rhs(int n1, int n2, typename Prec<MODE>::R ihx, typename Prec<MODE>::R ihz,
                                               const RIN* __restrict__ r, const typename Prec<MODE>::V* __restrict__ ep,
                                               typename Prec<MODE>::V* su1, typename Prec<MODE>::V* su2, RhsStride rs) {
    pdl_prologue();
    using V = typename Prec<MODE>::V;
    using R = typename Prec<MODE>::R;
    const int np = n1 * n2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int rr = blockIdx.y;
    if (t >= np || (rs.active && !rs.active[rr])) return;
    r += rr * rs.s0;
    ep += rr * rs.s1;
    su1 += rr * rs.s2;
    su2 += rr * rs.s2;
    const int i = t % n1, j = t / n1;
    const V e = ep[t];
    V s1 = czero<V>(), s2 = czero<V>();
    if (i >= 1) {
        const auto rv = InLoad<R>::get(r, t);
        V ew = ep[t - 1];
        s1 = cmk<V>((R)rv.x - ihx * (e.x - ew.x), (R)rv.y - ihx * (e.y - ew.y));
    }
    if (j >= 1) {
        const auto rv = InLoad<R>::get(r, np + t);
        V es = ep[t - n1];
        s2 = cmk<V>((R)rv.x - ihz * (e.x - es.x), (R)rv.y - ihz * (e.y - es.y));
    }
    su1[t] = s1;
    su2[t] = s2;
}

template <int MODE, class RIN>
void launch_u_rhs(int n1, int n2, double ihx, double ihz, const RIN* r, const typename Prec<MODE>::V* ep,
                  typename Prec<MODE>::V* su1, typename Prec<MODE>::V* su2, cudaStream_t st, int nrhs, RhsStride rs) {
    int np = n1 * n2;
    launch_pdl(k_u_rhs<MODE, RIN>, dim3(dim3((np + 255) / 256, nrhs)), dim3(256), 0, st, n1, n2, (typename Prec<MODE>::R)ihx,
                                                                 (typename Prec<MODE>::R)ihz, r, ep, su1, su2, rs);
}
template void launch_u_rhs<BAH_FP64, double2>(int, int, double, double, const double2*, const double2*, double2*,
                                              double2*, cudaStream_t, int, RhsStride);
template void launch_u_rhs<BAH_MIXED, double2>(int, int, double, double, const double2*, const float2*, float2*,
                                               float2*, cudaStream_t, int, RhsStride);
template void launch_u_rhs<BAH_FP64, float4>(int, int, double, double, const float4*, const double2*, double2*,
                                             double2*, cudaStream_t, int, RhsStride);
template void launch_u_rhs<BAH_MIXED, float4>(int, int, double, double, const float4*, const float2*, float2*,
                                              float2*, cudaStream_t, int, RhsStride);

// ---------------------------------------------------------------------------
// element-wise precision conversion
// ---------------------------------------------------------------------------
template <class Vin, class Vout>
__global__ void k_convert(const Vin* __restrict__ x, Vout* __restrict__ y, size_t n) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n) y[t] = cconv<Vout>(x[t]);
}
template <class Vin, class Vout>
void launch_convert(const Vin* x, Vout* y, size_t n, cudaStream_t st) {
    k_convert<Vin, Vout><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
}
template void launch_convert<double2, float2>(const double2*, float2*, size_t, cudaStream_t);
template void launch_convert<float2, double2>(const float2*, double2*, size_t, cudaStream_t);
template void launch_convert<double2, double2>(const double2*, double2*, size_t, cudaStream_t);

// ---------------------------------------------------------------------------
// zero the boundary-normal (non-unknown) entries of padded vectors
// ---------------------------------------------------------------------------
__global__ void k_sanitize(double2* v, int n1, int n2, int nvec) {
    const int np = n1 * n2;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)np * nvec) return;
    const int k = (int)(t / np), pt = (int)(t % np);
    const int i = pt % n1, j = pt / n1;
    double2* u = v + (size_t)k * 3 * np;
    if (i == 0) u[pt] = make_double2(0.0, 0.0);
    if (j == 0) u[np + pt] = make_double2(0.0, 0.0);
}
void launch_sanitize(double2* v, int n1, int n2, int nvec, cudaStream_t st) {
    size_t n = (size_t)n1 * n2 * nvec;
    k_sanitize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, n1, n2, nvec);
}

}  // namespace bah
