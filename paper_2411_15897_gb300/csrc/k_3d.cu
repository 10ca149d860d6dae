// Three-dimensional grids: the mixed elastic operator (Eq. 2.6), the
// distributor and back-substitution of the block-acoustic preconditioner
// (Eq. 3.3 - 3.5), and the multigrid of its four acoustic blocks (Sec. 2.2;
// Galerkin coarsening, Eq. 4.3, with the mixed intergrid of Eq. 4.4, the
// transfer the paper takes for its 3-D experiments, Sec. 4.5).
//
// Point (i, j, k) of an n1 x n2 x n3 grid sits at (k*n2 + j)*n1 + i.  Every
// block lives on the padded index space of its level: block type a < 3
// (u_{a+1}, nodal along x_{a+1}) has unknowns where that coordinate is >= 1,
// type 3 (p) at every point; the other points hold structural zeros, which
// every kernel writes as zero and none reads as an unknown.
//
// Each kernel runs one thread per point and bounds-checks every neighbour
// against the grid before it loads it.  The kernels of the solve's step begin
// with pdl_prologue() and are launched with programmatic dependent launch; the
// level kernels run the three displacement blocks of a level in one launch.
#include "bah_internal.cuh"

#include <type_traits>

namespace bah {

// pointers of up to three blocks of one level, one per blockIdx.y of a launch;
// pick() selects without indexing the parameter array at a run-time index
// (which would copy it to the stack)
template <class T> struct Set3 { T* p[3]; };
template <class T> __device__ __forceinline__ T* pick(const Set3<T>& s, int y) {
    return y == 0 ? s.p[0] : (y == 1 ? s.p[1] : s.p[2]);
}

__host__ __device__ __forceinline__ bool valid3(int type, const int* c) { return type >= 3 || c[type] >= 1; }

__device__ __forceinline__ void coords3(int p, int n1, int n2, int* c) {
    c[0] = p % n1;
    const int t = p / n1;
    c[1] = t % n2;
    c[2] = t / n2;
}

// stencil entry s -> offset: 7-point (0 centre, 1 + 2a at -e_a, 2 + 2a at +e_a)
// or 27-point ((dz+1)*9 + (dy+1)*3 + (dx+1))
template <int NS> __host__ __device__ __forceinline__ void soff(int s, int* o) {
    if (NS == 7) {
        o[0] = o[1] = o[2] = 0;
        if (s > 0) o[(s - 1) >> 1] = ((s - 1) & 1) ? 1 : -1;
    } else {
        o[0] = s % 3 - 1;
        o[1] = (s / 3) % 3 - 1;
        o[2] = s / 9 - 1;
    }
}
template <int NS> __host__ __device__ constexpr int scentre() { return NS == 7 ? 0 : 13; }

// ---------------------------------------------------------------------------
// medium: 1/(lambda+mu), omega^2 rho~ (rho~ = rho (1 - i gamma/omega)) and
// the edge means of mu.  mue[e] belongs to the pair of axes other than e; at a
// point whose coordinates along that pair are (a, b) it is the mean of mu over
// the four cells around the edge at nodes (a, b), zero on boundary edges
// (where the tangential derivative is dropped with the zero normal
// displacement), the same averaging as the 2-D operator's nodes.
// ---------------------------------------------------------------------------
__global__ void k_prep3_cells(int n1, int n2, int n3, double omega, const double* __restrict__ lam,
                              const double* __restrict__ mu, const double* __restrict__ rho,
                              const double* __restrict__ gam, double* cinv, double2* mrt, double* mue0, double* mue1,
                              double* mue2) {
    const int np = n1 * n2 * n3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    coords3(p, n1, n2, c);
    const int st[3] = {1, n1, n1 * n2};
    cinv[p] = 1.0 / (lam[p] + mu[p]);
    mrt[p] = make_double2(omega * omega * rho[p], -omega * rho[p] * gam[p]);
    double* mue[3] = {mue0, mue1, mue2};
    for (int e = 0; e < 3; ++e) {
        const int a = e == 0 ? 1 : 0, b = e == 2 ? 1 : 2;
        double v = 0.0;
        if (c[a] >= 1 && c[b] >= 1)
            v = 0.25 * (mu[p] + mu[p - st[a]] + mu[p - st[b]] + mu[p - st[a] - st[b]]);
        mue[e][p] = v;
    }
}

// diagonals of A_a (unshifted) and the FP64 7-point fine stencils of the four
// shifted blocks A_{a,s} (Eq. 2.6 with the shift of Eq. 2.8) and H_{p,s}
// (Eq. 3.4: B B^T diag((lambda+2mu)/(lambda+mu)) - omega^2 diag(rho~/(lambda+mu)),
// shifted by i alpha omega^2 rho/(lambda+mu))
__global__ void k_prep3_blocks(Op3 op, double alpha, double omega, const double* __restrict__ rho,
                               const double* __restrict__ mu, double2* dg0, double2* dg1, double2* dg2,
                               double2* S0, double2* S1, double2* S2, double2* S3) {
    const int n1 = op.n[0], n2 = op.n[1], n3 = op.n[2];
    const int np = n1 * n2 * n3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    coords3(p, n1, n2, c);
    const int st[3] = {1, n1, n1 * n2};
    double2* dg[3] = {dg0, dg1, dg2};
    double2* S[4] = {S0, S1, S2, S3};
    const double aw2 = alpha * omega * omega;
    for (int a = 0; a < 3; ++a) {
        double2 e[7];
        for (int s = 0; s < 7; ++s) e[s] = make_double2(0.0, 0.0);
        double2 d = make_double2(0.0, 0.0);
        if (c[a] >= 1) {
            const int pm = p - st[a];
            double dr = op.ih2[a] * (mu[pm] + mu[p]);
            if (c[a] >= 2) e[1 + 2 * a].x = -op.ih2[a] * mu[pm];
            if (c[a] + 1 <= op.n[a] - 1) e[2 + 2 * a].x = -op.ih2[a] * mu[p];
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                const double* me = op.mue[3 - a - b];
                const double lo = c[b] >= 1 ? me[p] : 0.0;
                const double hi = c[b] + 1 <= op.n[b] - 1 ? me[p + st[b]] : 0.0;
                dr += op.ih2[b] * (lo + hi);
                e[1 + 2 * b].x = -op.ih2[b] * lo;
                e[2 + 2 * b].x = -op.ih2[b] * hi;
            }
            const double2 m = make_double2(0.5 * (op.mrt[pm].x + op.mrt[p].x), 0.5 * (op.mrt[pm].y + op.mrt[p].y));
            d = make_double2(dr - m.x, -m.y);
            e[0] = make_double2(d.x, d.y + aw2 * 0.5 * (rho[pm] + rho[p]));
        }
        dg[a][p] = d;
        for (int s = 0; s < 7; ++s) S[a][(size_t)s * np + p] = e[s];
    }
    // H_p,s
    {
        double2 e[7];
        for (int s = 0; s < 7; ++s) e[s] = make_double2(0.0, 0.0);
        const double wp = 1.0 + mu[p] * op.cinv[p];
        double cen = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (c[a] >= 1) {
                const int q = p - st[a];
                cen += op.ih2[a] * wp;
                e[1 + 2 * a].x = -op.ih2[a] * (1.0 + mu[q] * op.cinv[q]);
            }
            if (c[a] + 1 <= op.n[a] - 1) {
                const int q = p + st[a];
                cen += op.ih2[a] * wp;
                e[2 + 2 * a].x = -op.ih2[a] * (1.0 + mu[q] * op.cinv[q]);
            }
        }
        e[0] = make_double2(cen - op.mrt[p].x * op.cinv[p], -op.mrt[p].y * op.cinv[p] + aw2 * rho[p] * op.cinv[p]);
        for (int s = 0; s < 7; ++s) S[3][(size_t)s * np + p] = e[s];
    }
}

void launch_prep3(const Op3& op, double omega, double alpha, const double* lam, const double* mu, const double* rho,
                  const double* gam, double* cinv, double2* mrt, double* const* mue, double2* const* dg,
                  double2* const* S, cudaStream_t st) {
    const int np = op.n[0] * op.n[1] * op.n[2];
    const int nb = (np + 255) / 256;
    k_prep3_cells<<<nb, 256, 0, st>>>(op.n[0], op.n[1], op.n[2], omega, lam, mu, rho, gam, cinv, mrt, mue[0], mue[1],
                                      mue[2]);
    k_prep3_blocks<<<nb, 256, 0, st>>>(op, alpha, omega, rho, mu, dg[0], dg[1], dg[2], S[0], S[1], S[2], S[3]);
}

// ---------------------------------------------------------------------------
// y = H x (Eq. 2.6), y = b - H x with b, or y = H^H x = conj(H) x (H is complex
// symmetric; only the mass diagonals are complex).  Right-hand side r of the
// launch is blockIdx.y, at element strides sx, sy, sb.
// ---------------------------------------------------------------------------
template <class Vin>
__global__ void __launch_bounds__(256) k_apply3(Op3 op, const Vin* __restrict__ x, double2* __restrict__ y,
                                                const double2* __restrict__ b, int conj, size_t sx, size_t sy,
                                                size_t sb) {
    pdl_prologue();
    const int n1 = op.n[0], n2 = op.n[1];
    const int np = n1 * n2 * op.n[2];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    x += blockIdx.y * sx;
    y += blockIdx.y * sy;
    if (b) b += blockIdx.y * sb;
    int c[3];
    coords3(p, n1, n2, c);
    const int st[3] = {1, n1, n1 * n2};
    auto ld = [&](int comp, int q) { return cconv<double2>(x[(size_t)comp * np + q]); };
    const double2 pc = ld(3, p);
    double2 out[4];
    for (int a = 0; a < 3; ++a) {
        if (c[a] == 0) { out[a] = make_double2(0.0, 0.0); continue; }
        double2 d = op.dg[a][p];
        if (conj) d.y = -d.y;
        double2 acc = cmul(d, ld(a, p));
        const int pm = p - st[a];
        if (c[a] >= 2) acc = csub(acc, cscale(ld(a, pm), op.ih2[a] * op.muc[pm]));
        if (c[a] + 1 <= op.n[a] - 1) acc = csub(acc, cscale(ld(a, p + st[a]), op.ih2[a] * op.muc[p]));
        for (int bb = 0; bb < 3; ++bb) {
            if (bb == a) continue;
            const double* me = op.mue[3 - a - bb];
            if (c[bb] >= 1) acc = csub(acc, cscale(ld(a, p - st[bb]), op.ih2[bb] * me[p]));
            if (c[bb] + 1 <= op.n[bb] - 1) acc = csub(acc, cscale(ld(a, p + st[bb]), op.ih2[bb] * me[p + st[bb]]));
        }
        acc = cadd(acc, cscale(csub(pc, ld(3, pm)), op.ih[a]));
        out[a] = acc;
    }
    {
        double2 acc = cscale(pc, -op.cinv[p]);
        for (int a = 0; a < 3; ++a) {
            if (c[a] >= 1) acc = cadd(acc, cscale(ld(a, p), op.ih[a]));
            if (c[a] + 1 <= op.n[a] - 1) acc = csub(acc, cscale(ld(a, p + st[a]), op.ih[a]));
        }
        out[3] = acc;
    }
    for (int k = 0; k < 4; ++k) {
        const bool v = k == 3 || c[k] >= 1;
        double2 o = out[k];
        if (b && v) o = csub(b[(size_t)k * np + p], o);
        y[(size_t)k * np + p] = v ? o : make_double2(0.0, 0.0);
    }
}

template <class Vin>
void launch_apply3(const Op3& op, const Vin* x, double2* y, const double2* b, int conj, int nrhs, size_t sx, size_t sy,
                   size_t sb, cudaStream_t st) {
    const int np = op.n[0] * op.n[1] * op.n[2];
    if (nrhs < 1) return;
    launch_pdl(k_apply3<Vin>, dim3((np + 255) / 256, nrhs), dim3(256), 0, st, op, x, y, b, conj, sx, sy, sb);
}
template void launch_apply3<double2>(const Op3&, const double2*, double2*, const double2*, int, int, size_t, size_t,
                                     size_t, cudaStream_t);
template void launch_apply3<float2>(const Op3&, const float2*, double2*, const double2*, int, int, size_t, size_t,
                                    size_t, cudaStream_t);

// zero the boundary-normal entries of nvec padded vectors
__global__ void k_sanitize3(double2* v, int n1, int n2, int n3, int nvec) {
    const int np = n1 * n2 * n3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    coords3(p, n1, n2, c);
    for (int r = 0; r < nvec; ++r)
        for (int a = 0; a < 3; ++a)
            if (c[a] == 0) v[((size_t)r * 4 + a) * np + p] = make_double2(0.0, 0.0);
}
void launch_sanitize3(double2* v, int n1, int n2, int n3, int nvec, cudaStream_t st) {
    const int np = n1 * n2 * n3;
    k_sanitize3<<<(np + 255) / 256, 256, 0, st>>>(v, n1, n2, n3, nvec);
}

// ---------------------------------------------------------------------------
// distributor (Eq. 3.3, second row): t_p = B r_u - A_p r_p with
// A_p = B B^T diag(mu) - omega^2 diag(rho~) (Eq. 3.2); FP64 arithmetic,
// result in the cycle's vector type
// ---------------------------------------------------------------------------
template <class V>
__global__ void __launch_bounds__(256) k_distrib3(Op3 op, const double2* __restrict__ r, V* __restrict__ tp) {
    pdl_prologue();
    const int n1 = op.n[0], n2 = op.n[1];
    const int np = n1 * n2 * op.n[2];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    coords3(p, n1, n2, c);
    const int st[3] = {1, n1, n1 * n2};
    const double2* rp = r + (size_t)3 * np;
    const double2 mrp = cscale(rp[p], op.muc[p]);
    double2 acc = cmul(op.mrt[p], rp[p]);        // + omega^2 rho~ r_p
    for (int a = 0; a < 3; ++a) {
        const double2* ra = r + (size_t)a * np;
        if (c[a] >= 1) {
            const int q = p - st[a];
            acc = cadd(acc, cscale(ra[p], op.ih[a]));
            acc = csub(acc, cscale(csub(mrp, cscale(rp[q], op.muc[q])), op.ih2[a]));
        }
        if (c[a] + 1 <= op.n[a] - 1) {
            const int q = p + st[a];
            acc = csub(acc, cscale(ra[q], op.ih[a]));
            acc = csub(acc, cscale(csub(mrp, cscale(rp[q], op.muc[q])), op.ih2[a]));
        }
    }
    tp[p] = cconv<V>(acc);
}

// back-substitution (Eq. 3.5): s_a = r_a - (B^T e_p)_a for the three u blocks
template <class V>
__global__ void __launch_bounds__(256) k_urhs3(Op3 op, const double2* __restrict__ r, const V* __restrict__ ep,
                                               V* __restrict__ s0, V* __restrict__ s1, V* __restrict__ s2) {
    pdl_prologue();
    const int n1 = op.n[0], n2 = op.n[1];
    const int np = n1 * n2 * op.n[2];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    coords3(p, n1, n2, c);
    const int st[3] = {1, n1, n1 * n2};
    V* s[3] = {s0, s1, s2};
    const double2 e0 = cconv<double2>(ep[p]);
    for (int a = 0; a < 3; ++a) {
        double2 v = make_double2(0.0, 0.0);
        if (c[a] >= 1) {
            const double2 g = cscale(csub(e0, cconv<double2>(ep[p - st[a]])), op.ih[a]);
            v = csub(r[(size_t)a * np + p], g);
        }
        s[a][p] = cconv<V>(v);
    }
}

template <class V>
void launch_distrib3(const Op3& op, const double2* r, V* tp, cudaStream_t st) {
    const int np = op.n[0] * op.n[1] * op.n[2];
    launch_pdl(k_distrib3<V>, dim3((np + 255) / 256), dim3(256), 0, st, op, r, tp);
}
template <class V>
void launch_urhs3(const Op3& op, const double2* r, const V* ep, V* const* su, cudaStream_t st) {
    const int np = op.n[0] * op.n[1] * op.n[2];
    launch_pdl(k_urhs3<V>, dim3((np + 255) / 256), dim3(256), 0, st, op, r, ep, su[0], su[1], su[2]);
}
template void launch_distrib3<double2>(const Op3&, const double2*, double2*, cudaStream_t);
template void launch_distrib3<float2>(const Op3&, const double2*, float2*, cudaStream_t);
template void launch_urhs3<double2>(const Op3&, const double2*, const double2*, double2* const*, cudaStream_t);
template void launch_urhs3<float2>(const Op3&, const double2*, const float2*, float2* const*, cudaStream_t);

// ---------------------------------------------------------------------------
// multigrid level kernels.  Stencils are stored entry-major: entry s of
// point p at S[s * points + p].
// ---------------------------------------------------------------------------
// one damped Jacobi sweep x_out = x_in + w D^{-1} (b - A x_in) (zero: x_in = 0),
// or the residual x_out = b - A x_in (res), for up to three blocks of one
// level in one launch: blockIdx.y = y runs block type type0 + y on the y-th
// pointers.  Stencil entries are stored as SC: FP64 complex, or bfloat16
// complex in mixed mode, where every entry and neighbour of a point is loaded
// before the first multiply-add.
template <class V, class SC, int NS>
__global__ void __launch_bounds__(256) k_jacobi3(int type0, int n1, int n2, int n3, Set3<const SC> Sset,
                                                 Set3<const V> bset, Set3<const V> xiset, Set3<V> xoset,
                                                 typename VecTraits<V>::R w, int zero, int res) {
    pdl_prologue();
    const int y = blockIdx.y, type = type0 + y;
    const SC* __restrict__ S = pick(Sset, y);
    const V* __restrict__ b = pick(bset, y);
    const V* xin = pick(xiset, y);
    V* xout = pick(xoset, y);
    const int np = n1 * n2 * n3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int c[3];
    coords3(p, n1, n2, c);
    if (!valid3(type, c)) { xout[p] = czero<V>(); return; }
    const int n[3] = {n1, n2, n3};
    const int st[3] = {1, n1, n1 * n2};
    V acc = b[p];
    if (!zero) {
        constexpr bool kBatch = sizeof(SC) <= 4;          // bf16 entries: all loads first
        SC sv[kBatch ? NS : 1];
        V xv[kBatch ? NS : 1];
        bool inn[kBatch ? NS : 1];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            int o[3];
            soff<NS>(s, o);
            bool in = true;
            int q = p;
            for (int a = 0; a < 3; ++a) {
                const int cc = c[a] + o[a];
                if (cc < 0 || cc >= n[a]) in = false;
                q += o[a] * st[a];
            }
            if constexpr (kBatch) {
                inn[s] = in;
                sv[s] = S[(size_t)s * np + p];
                xv[s] = xin[in ? q : p];
            } else {
                if (in) acc = csub(acc, cmul(ldc(S[(size_t)s * np + p]), xin[q]));
            }
        }
        if constexpr (kBatch) {
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (inn[s]) acc = csub(acc, cmul(ldc(sv[s]), xv[s]));
        }
    }
    if (res) { xout[p] = acc; return; }
    const V upd = cscale(cdiv(acc, ldc(S[(size_t)scentre<NS>() * np + p])), w);
    xout[p] = zero ? upd : cadd(xin[p], upd);
}

template <class T>
static Set3<T> set3(T* const* v, int nq) {
    Set3<T> s;
    for (int y = 0; y < 3; ++y) s.p[y] = y < nq ? v[y] : nullptr;
    return s;
}

template <class V>
void launch_jacobi3(int type0, int nq, const int* n, int ns, const void* const* S, const V* const* b,
                    const V* const* xin, V* const* xout, double w, int zero, int res, cudaStream_t st) {
    const int np = n[0] * n[1] * n[2];
    using R = typename VecTraits<V>::R;
    using SC = typename std::conditional<std::is_same<V, double2>::value, double2, __nv_bfloat162>::type;
    const SC* s[3];
    for (int y = 0; y < nq; ++y) s[y] = (const SC*)S[y];
    const Set3<const SC> ss = set3<const SC>(s, nq);
    const dim3 g((np + 255) / 256, nq);
    if (ns == 7)
        launch_pdl(k_jacobi3<V, SC, 7>, g, dim3(256), 0, st, type0, n[0], n[1], n[2], ss, set3<const V>(b, nq),
                   set3<const V>(xin, nq), set3<V>(xout, nq), (R)w, zero, res);
    else
        launch_pdl(k_jacobi3<V, SC, 27>, g, dim3(256), 0, st, type0, n[0], n[1], n[2], ss, set3<const V>(b, nq),
                   set3<const V>(xin, nq), set3<V>(xout, nq), (R)w, zero, res);
}
template void launch_jacobi3<double2>(int, int, const int*, int, const void* const*, const double2* const*,
                                      const double2* const*, double2* const*, double, int, int, cudaStream_t);
template void launch_jacobi3<float2>(int, int, const int*, int, const void* const*, const float2* const*,
                                     const float2* const*, float2* const*, double, int, int, cudaStream_t);

// 1-D transfer weights.  Restriction (Eq. 4.1 / 4.4, mixed intergrid): along
// the block's nodal axis 1/4 [1 2 1] around fine face 2K; along a cell-centred
// axis 1/2 [1 1] over fine cells 2J, 2J+1.  Prolongation: linear interpolation
// along the nodal axis (missing coarse faces are the zero boundary) and
// bilinear cell-centred interpolation with constant extrapolation at the ends.
__host__ __device__ __forceinline__ int rlist3(bool nodal, int J, int* f, double* w) {
    if (nodal) {
        f[0] = 2 * J - 1; w[0] = 0.25;
        f[1] = 2 * J;     w[1] = 0.5;
        f[2] = 2 * J + 1; w[2] = 0.25;
        return 3;
    }
    f[0] = 2 * J;     w[0] = 0.5;
    f[1] = 2 * J + 1; w[1] = 0.5;
    return 2;
}
__host__ __device__ __forceinline__ int plist3(bool nodal, int m, int nc, int* K, double* w) {
    if (nodal) {
        if ((m & 1) == 0) {
            K[0] = m >> 1; w[0] = 1.0;
            return (K[0] >= 1 && K[0] <= nc - 1) ? 1 : 0;
        }
        int cnt = 0;
        if (((m - 1) >> 1) >= 1) { K[cnt] = (m - 1) >> 1; w[cnt++] = 0.5; }
        if (((m + 1) >> 1) <= nc - 1) { K[cnt] = (m + 1) >> 1; w[cnt++] = 0.5; }
        return cnt;
    }
    const int J = m >> 1;
    int Jn = (m & 1) ? J + 1 : J - 1;
    if (Jn < 0 || Jn > nc - 1) Jn = J;
    K[0] = J;  w[0] = 0.75;
    K[1] = Jn; w[1] = 0.25;
    return 2;
}

// the transfer weights of one axis as a fixed number of (index, weight)
// pairs, unused pairs with weight 0 at an in-range index, so that the
// kernels below keep them in registers: restriction, three fine indices;
// prolongation, two coarse indices (the same weights as rlist3 / plist3)
template <class R>
__device__ __forceinline__ void raxis3(bool nodal, int J, int* f, R* w) {
    if (nodal) {
        f[0] = 2 * J - 1; w[0] = R(0.25);
        f[1] = 2 * J;     w[1] = R(0.5);
        f[2] = 2 * J + 1; w[2] = R(0.25);
    } else {
        f[0] = 2 * J;     w[0] = R(0.5);
        f[1] = 2 * J + 1; w[1] = R(0.5);
        f[2] = 2 * J;     w[2] = R(0);
    }
}
template <class R>
__device__ __forceinline__ void paxis3(bool nodal, int m, int nc, int* K, R* w) {
    if (nodal) {
        if ((m & 1) == 0) {
            K[0] = m >> 1; w[0] = (K[0] >= 1 && K[0] <= nc - 1) ? R(1) : R(0);
            K[1] = K[0];   w[1] = R(0);
        } else {
            K[0] = (m - 1) >> 1; w[0] = K[0] >= 1 ? R(0.5) : R(0);
            K[1] = (m + 1) >> 1; w[1] = K[1] <= nc - 1 ? R(0.5) : R(0);
        }
        K[0] = min(K[0], nc - 1);
        K[1] = min(K[1], nc - 1);
        return;
    }
    const int J = m >> 1;
    int Jn = (m & 1) ? J + 1 : J - 1;
    if (Jn < 0 || Jn > nc - 1) Jn = J;
    K[0] = J;  w[0] = R(0.75);
    K[1] = Jn; w[1] = R(0.25);
}

// b_c = R r on the coarse grid (fine grid n, coarse n/2), accumulated in the
// cycle's arithmetic (FP32 in mixed mode; the weights 1/2 and 1/4 and their
// products are exact there)
template <class V>
__global__ void __launch_bounds__(256) k_restrict3(int type0, int f1, int f2, int f3, Set3<const V> rset,
                                                   Set3<V> bcset) {
    pdl_prologue();
    const int type = type0 + (int)blockIdx.y;
    const V* __restrict__ r = pick(rset, (int)blockIdx.y);
    V* __restrict__ bc = pick(bcset, (int)blockIdx.y);
    const int c1 = f1 / 2, c2 = f2 / 2, c3 = f3 / 2;
    const int npc = c1 * c2 * c3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npc) return;
    int J[3];
    coords3(p, c1, c2, J);
    if (!valid3(type, J)) { bc[p] = czero<V>(); return; }
    using R = typename VecTraits<V>::R;
    int fx[3], fy[3], fz[3];
    R wx[3], wy[3], wz[3];
    raxis3<R>(type == 0, J[0], fx, wx);
    raxis3<R>(type == 1, J[1], fy, wy);
    raxis3<R>(type == 2, J[2], fz, wz);
    V acc = czero<V>();
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const R wzy = wz[z] * wy[y];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const R ww = wzy * wx[x];
                if (ww != R(0)) {
                    const V v = r[((size_t)fz[z] * f2 + fy[y]) * f1 + fx[x]];
                    acc.x += ww * v.x;
                    acc.y += ww * v.y;
                }
            }
        }
    bc[p] = acc;
}

// x += P e_c on the fine grid
template <class V>
__global__ void __launch_bounds__(256) k_prolong3(int type0, int f1, int f2, int f3, Set3<const V> ecset,
                                                  Set3<V> xset) {
    pdl_prologue();
    const int type = type0 + (int)blockIdx.y;
    const V* __restrict__ ec = pick(ecset, (int)blockIdx.y);
    V* __restrict__ x = pick(xset, (int)blockIdx.y);
    const int c1 = f1 / 2, c2 = f2 / 2, c3 = f3 / 2;
    const int np = f1 * f2 * f3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    int F[3];
    coords3(p, f1, f2, F);
    if (!valid3(type, F)) return;
    using R = typename VecTraits<V>::R;
    int kx[2], ky[2], kz[2];
    R wx[2], wy[2], wz[2];
    paxis3<R>(type == 0, F[0], c1, kx, wx);
    paxis3<R>(type == 1, F[1], c2, ky, wy);
    paxis3<R>(type == 2, F[2], c3, kz, wz);
    V acc = czero<V>();
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const R wzy = wz[z] * wy[y];
#pragma unroll
            for (int xx = 0; xx < 2; ++xx) {
                const R ww = wzy * wx[xx];
                if (ww != R(0)) {
                    const V v = ec[((size_t)kz[z] * c2 + ky[y]) * c1 + kx[xx]];
                    acc.x += ww * v.x;
                    acc.y += ww * v.y;
                }
            }
        }
    x[p] = cadd(x[p], acc);
}

template <class V>
void launch_restrict3(int type0, int nq, const int* nf, const V* const* r, V* const* bc, cudaStream_t st) {
    const int npc = (nf[0] / 2) * (nf[1] / 2) * (nf[2] / 2);
    launch_pdl(k_restrict3<V>, dim3((npc + 255) / 256, nq), dim3(256), 0, st, type0, nf[0], nf[1], nf[2],
               set3<const V>(r, nq), set3<V>(bc, nq));
}
template <class V>
void launch_prolong3(int type0, int nq, const int* nf, const V* const* ec, V* const* x, cudaStream_t st) {
    const int np = nf[0] * nf[1] * nf[2];
    launch_pdl(k_prolong3<V>, dim3((np + 255) / 256, nq), dim3(256), 0, st, type0, nf[0], nf[1], nf[2],
               set3<const V>(ec, nq), set3<V>(x, nq));
}
template void launch_restrict3<double2>(int, int, const int*, const double2* const*, double2* const*, cudaStream_t);
template void launch_restrict3<float2>(int, int, const int*, const float2* const*, float2* const*, cudaStream_t);
template void launch_prolong3<double2>(int, int, const int*, const double2* const*, double2* const*, cudaStream_t);
template void launch_prolong3<float2>(int, int, const int*, const float2* const*, float2* const*, cudaStream_t);

// ---------------------------------------------------------------------------
// Galerkin coarse operator A_c = R A P (Eq. 4.3) in FP64, one thread per
// coarse point, from a 7- or 27-point fine stencil to a 27-point coarse one.
// With the mixed intergrid every coarse coupling stays within one point per
// axis; a coupling outside sets *err (it would mean a wrong transfer).
// ---------------------------------------------------------------------------
template <int NSF>
__global__ void k_galerkin3(int type, int f1, int f2, int f3, const double2* __restrict__ Sf, double2* __restrict__ Sc,
                            int* err) {
    const int nc[3] = {f1 / 2, f2 / 2, f3 / 2};
    const int nf[3] = {f1, f2, f3};
    const int npc = nc[0] * nc[1] * nc[2];
    const int npf = f1 * f2 * f3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npc) return;
    int J[3];
    coords3(p, nc[0], nc[1], J);
    double2 acc[27];
    for (int s = 0; s < 27; ++s) acc[s] = make_double2(0.0, 0.0);
    if (valid3(type, J)) {
        int f[3][3], cnt[3];
        double wr[3][3];
        for (int a = 0; a < 3; ++a) cnt[a] = rlist3(a == type, J[a], f[a], wr[a]);
        for (int z = 0; z < cnt[2]; ++z)
            for (int y = 0; y < cnt[1]; ++y)
                for (int x = 0; x < cnt[0]; ++x) {
                    const int A[3] = {f[0][x], f[1][y], f[2][z]};
                    const double w0 = wr[0][x] * wr[1][y] * wr[2][z];
                    const size_t pa = ((size_t)A[2] * f2 + A[1]) * f1 + A[0];
                    for (int s = 0; s < NSF; ++s) {
                        int o[3];
                        soff<NSF>(s, o);
                        int B[3];
                        bool in = true;
                        for (int a = 0; a < 3; ++a) {
                            B[a] = A[a] + o[a];
                            if (B[a] < 0 || B[a] >= nf[a]) in = false;
                        }
                        if (!in) continue;
                        const double2 v = Sf[(size_t)s * npf + pa];
                        if (v.x == 0.0 && v.y == 0.0) continue;
                        int K[3][2], pc[3];
                        double wp[3][2];
                        for (int a = 0; a < 3; ++a) pc[a] = plist3(a == type, B[a], nc[a], K[a], wp[a]);
                        for (int kz = 0; kz < pc[2]; ++kz)
                            for (int ky = 0; ky < pc[1]; ++ky)
                                for (int kx = 0; kx < pc[0]; ++kx) {
                                    const int d0 = K[0][kx] - J[0], d1 = K[1][ky] - J[1], d2 = K[2][kz] - J[2];
                                    if (d0 < -1 || d0 > 1 || d1 < -1 || d1 > 1 || d2 < -1 || d2 > 1) {
                                        *err = 1;
                                        continue;
                                    }
                                    const double ww = w0 * wp[0][kx] * wp[1][ky] * wp[2][kz];
                                    double2& t = acc[(d2 + 1) * 9 + (d1 + 1) * 3 + (d0 + 1)];
                                    t.x += ww * v.x;
                                    t.y += ww * v.y;
                                }
                    }
                }
    }
    for (int s = 0; s < 27; ++s) Sc[(size_t)s * npc + p] = acc[s];
}

void launch_galerkin3(int type, const int* nf, int nsf, const double2* Sf, double2* Sc, int* err, cudaStream_t st) {
    const int npc = (nf[0] / 2) * (nf[1] / 2) * (nf[2] / 2);
    if (nsf == 7)
        k_galerkin3<7><<<(npc + 127) / 128, 128, 0, st>>>(type, nf[0], nf[1], nf[2], Sf, Sc, err);
    else
        k_galerkin3<27><<<(npc + 127) / 128, 128, 0, st>>>(type, nf[0], nf[1], nf[2], Sf, Sc, err);
}

// dense matrix of the coarsest 27-point stencil over all points (identity
// rows at structural zeros) and X = I, for the Gauss-Jordan inverse
__global__ void k_dense_assemble3(int type, const double2* __restrict__ S, int n1, int n2, int n3, double2* A,
                                  double2* X) {
    const int np = n1 * n2 * n3;
    const int r = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= np || r >= np) return;
    int cr[3], cc[3];
    coords3(r, n1, n2, cr);
    coords3(col, n1, n2, cc);
    double2 v = make_double2(0.0, 0.0);
    if (valid3(type, cr)) {
        const int o0 = cc[0] - cr[0], o1 = cc[1] - cr[1], o2 = cc[2] - cr[2];
        if (o0 >= -1 && o0 <= 1 && o1 >= -1 && o1 <= 1 && o2 >= -1 && o2 <= 1)
            v = S[(size_t)((o2 + 1) * 9 + (o1 + 1) * 3 + (o0 + 1)) * np + r];
    } else if (col == r) {
        v = make_double2(1.0, 0.0);
    }
    A[(size_t)r * np + col] = v;
    X[(size_t)r * np + col] = make_double2(col == r ? 1.0 : 0.0, 0.0);
}

int coarse_invert3(int type, const int* n, const double2* S, double2* inv, double2* work, int* flag, cudaStream_t st) {
    const int np = n[0] * n[1] * n[2];
    if (np > 65535) {
        set_error("coarsest 3-D level too large for the dense inverse");
        return BAH_ERR_ARG;
    }
    dim3 g((np + 127) / 128, np);
    k_dense_assemble3<<<g, 128, 0, st>>>(type, S, n[0], n[1], n[2], work, inv);
    return gauss_jordan(np, work, inv, work + (size_t)np * np, flag, st);
}

}  // namespace bah
