// Shared-memory-resident multigrid on a thread-block cluster (mixed mode).
//
// The small levels of a block's hierarchy (here: every level from l0 down to
// the coarsest) are held entirely in the shared memory of one cluster of up
// to 16 CTAs, one CTA per SM.  Each level's grid rows are split into equal
// slabs, one per CTA; a CTA stores, for the points of its slab, the level's
// Galerkin stencil (bfloat16 complex, slot-major), the iterate, a work
// vector and the right-hand side.  The coarsest level is solved with the
// dense FP64 inverse, read from global memory (it stays in L2) and applied in
// FP64 arithmetic to the gathered FP32 right-hand side.  A stencil, restriction or prolongation tap
// that falls into another CTA's slab is read from that CTA's shared memory
// through the cluster's distributed shared memory (mapa + ld.shared::cluster).
//
// The cycle walks the same phases as the separate kernels -- zero-guess
// damped Jacobi, Jacobi, residual, restriction, the coarsest solve,
// prolongation and correction -- with the same per-point arithmetic, and the
// W-cycle's second coarse visits (Sec. 2.2), separated by the hardware
// cluster barrier.  Global memory is touched only to load the stencils and
// the level-l0 right-hand side (and iterate, on a warm start) at the start,
// to read the rows of the coarsest inverse, and to store the level-l0 result
// at the end.
//
// Deadlock freedom: the hardware co-schedules all CTAs of a cluster, every
// thread of every CTA executes the same sequence of barriers (the control
// flow depends only on kernel arguments; the only early exit is taken by a
// whole cluster at once), and a final barrier keeps every CTA's shared
// memory alive until no CTA of the cluster can still read it.
#include "bah_internal.cuh"
#include "intergrid.cuh"

#include <algorithm>
#include <cstring>

namespace bah {

constexpr int kSmThreads = 512;   // threads per CTA (one CTA per SM)

namespace {

__device__ __forceinline__ uint32_t mapa_rank(uint32_t local_addr, unsigned rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster_at(uint32_t cluster_addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(cluster_addr));
    return v;
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

}  // namespace

template <int RM>
__global__ void __launch_bounds__(kSmThreads, 1) k_cluster_mg(SmArgs a) {
    pdl_prologue();
    using V = float2;
    using CC = __nv_bfloat162;
    const unsigned cid = cluster_index();
    const int z = (int)(cid % (unsigned)a.nb), rr = (int)(cid / (unsigned)a.nb);
    if (a.active && !a.active[rr]) return;              // uniform over the cluster
    const unsigned q = cluster_rank();
    const int tid = threadIdx.x, nth = blockDim.x;
    const int type = a.b0 + z;
    const bool nodx = type == 0, nodz = type == 1;
    extern __shared__ __align__(16) unsigned char sm[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
    const int nlev = a.nlev, kc = nlev - 1;

    auto p0 = [&](const SmLevel& L) { return (int)q * L.rp * L.n1; };
    auto nown = [&](const SmLevel& L) {
        const int r0 = (int)q * L.rp, r1 = min(L.n2, r0 + L.rp);
        return r1 > r0 ? (r1 - r0) * L.n1 : 0;
    };
    auto vec = [&](unsigned off) { return reinterpret_cast<V*>(sm + off); };
    // cluster address of column 0 of grid row `row` of vector `off` of level L
    // (one owner lookup and one mapa per row; the columns follow at 8 bytes)
    auto row_addr = [&](const SmLevel& L, unsigned off, int row) -> uint32_t {
        const int owner = (int)(((float)row + 0.5f) * L.inv_rp);
        return mapa_rank(sbase + off + (uint32_t)((row - owner * L.rp) * L.n1) * 8u, (unsigned)owner);
    };
    // row and column of own point lt of level L
    auto own_rc = [&](const SmLevel& L, int lt, int& row, int& col) {
        const int r = (int)(((float)lt + 0.5f) * L.inv_n1);
        row = (int)q * L.rp + r;
        col = lt - r * L.n1;
    };
    auto coef = [&](int k) { return reinterpret_cast<const CC*>(sm + a.lv[k].off_c); };

    // ---- load: stencils, coarsest inverse rows, level-l0 vectors ----
    // asynchronous copies (cp.async), so that every thread keeps many loads in
    // flight; one wait for all of them before the first barrier
    for (int k = 0; k < kc; ++k) {
        const SmLevel& L = a.lv[k];
        const int np = L.n1 * L.n2, own = nown(L), g0 = p0(L), cap = L.rp * L.n1;
        const int nsl = (2 * a.rx[z][k] + 1) * (2 * a.rz[z][k] + 1);
        const CC* S = a.S[z][k];
        for (int s = 0; s < nsl; ++s)
            for (int t = tid; t < own; t += nth)
                cp_async4(sbase + L.off_c + (uint32_t)(s * cap + t) * 4u, S + (size_t)s * np + g0 + t);
    }
    {
        const SmLevel& L = a.lv[0];
        const int own = nown(L), g0 = p0(L);
        const size_t roff = (size_t)rr * L.n1 * L.n2 + g0;
        for (int t = tid; t < own; t += nth) {
            cp_async8(sbase + L.off_b + (uint32_t)t * 8u, a.gb[z] + roff + t);
            if (a.warm) cp_async8(sbase + L.off_x + (uint32_t)t * 8u, a.gx[z] + roff + t);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    cluster_barrier();

    // ---- phases (own points only; neighbours through distributed shared memory) ----
    auto stencil = [&](int k, unsigned xoff, int lt) -> V {
        const SmLevel& L = a.lv[k];
        const int rx = a.rx[z][k], rz = a.rz[z][k], wx = 2 * rx + 1, cap = L.rp * L.n1;
        int j, i;
        own_rc(L, lt, j, i);
        const CC* cs = coef(k);
        V sv[(2 * RM + 1) * (2 * RM + 1)], xv[(2 * RM + 1) * (2 * RM + 1)];
        bool in[(2 * RM + 1) * (2 * RM + 1)];
#pragma unroll
        for (int dz = -RM; dz <= RM; ++dz) {
            const int jj = j + dz;
            const bool rok = dz >= -rz && dz <= rz && jj >= 0 && jj < L.n2;
            const uint32_t ra = row_addr(L, xoff, rok ? jj : j);
#pragma unroll
            for (int dx = -RM; dx <= RM; ++dx) {
                const int qq = (dz + RM) * (2 * RM + 1) + (dx + RM);
                const int ii = i + dx;
                in[qq] = rok && dx >= -rx && dx <= rx && ii >= 0 && ii < L.n1;
                const int slot = in[qq] ? (dz + rz) * wx + (dx + rx) : 0;
                sv[qq] = ldc(cs[slot * cap + lt]);
                xv[qq] = ld_cluster_at(ra + (uint32_t)(in[qq] ? ii : i) * 8u);
            }
        }
        V acc = czero<V>();
#pragma unroll
        for (int e = 0; e < (2 * RM + 1) * (2 * RM + 1); ++e) {
            const float m = in[e] ? 1.f : 0.f;
            acc.x += m * (sv[e].x * xv[e].x - sv[e].y * xv[e].y);
            acc.y += m * (sv[e].x * xv[e].y + sv[e].y * xv[e].x);
        }
        return acc;
    };
    auto diag = [&](int k, int lt) -> V {
        const SmLevel& L = a.lv[k];
        const int rx = a.rx[z][k], rz = a.rz[z][k];
        return ldc(coef(k)[(rz * (2 * rx + 1) + rx) * (L.rp * L.n1) + lt]);
    };
    auto jacobi = [&](int k, unsigned xin, unsigned xout, bool zero) {
        const SmLevel& L = a.lv[k];
        const int own = nown(L);
        const V* b = vec(L.off_b);
        const V* xi = vec(xin);
        V* xo = vec(xout);
        for (int lt = tid; lt < own; lt += nth) {
            int j, i;
            own_rc(L, lt, j, i);
            if (!valid_pt(type, i, j)) { xo[lt] = czero<V>(); continue; }
            const V dg = diag(k, lt);
            if (zero) { xo[lt] = cscale(cdiv(b[lt], dg), L.w); continue; }
            const V ax = stencil(k, xin, lt);
            const V corr = cdiv(csub(b[lt], ax), dg);
            const V xv = xi[lt];
            xo[lt] = cmk<V>(xv.x + L.w * corr.x, xv.y + L.w * corr.y);
        }
    };
    auto residual = [&](int k, unsigned xin, unsigned rout) {
        const SmLevel& L = a.lv[k];
        const int own = nown(L);
        const V* b = vec(L.off_b);
        V* r = vec(rout);
        for (int lt = tid; lt < own; lt += nth) {
            int j, i;
            own_rc(L, lt, j, i);
            if (!valid_pt(type, i, j)) { r[lt] = czero<V>(); continue; }
            r[lt] = csub(b[lt], stencil(k, xin, lt));
        }
    };
    auto restrict_ = [&](int k, unsigned rin) {          // b_{k+1} = R r_k on own coarse points
        const SmLevel& L = a.lv[k];
        const SmLevel& Lc = a.lv[k + 1];
        const int own = nown(Lc);
        V* bc = vec(Lc.off_b);
        for (int lt = tid; lt < own; lt += nth) {
            int J, I;
            own_rc(Lc, lt, J, I);
            V acc = czero<V>();
            if (valid_pt(type, I, J)) {
                const int bx = rbase(nodx, a.intergrid, I), bz = rbase(nodz, a.intergrid, J);
                float wxs[4], wzs[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    wxs[e] = rw_axis_t<float>(nodx, a.intergrid, L.n1, I, bx + e);
                    wzs[e] = rw_axis_t<float>(nodz, a.intergrid, L.n2, J, bz + e);
                }
                V v[16];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool rok = wzs[e] != 0.f;
                    const uint32_t ra = row_addr(L, rin, rok ? bz + e : 0);
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const bool ok = rok && wxs[f] != 0.f;
                        v[e * 4 + f] = ld_cluster_at(ra + (uint32_t)(ok ? bx + f : 0) * 8u);
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const float wgt = wzs[e] * wxs[f];
                        acc.x += wgt * v[e * 4 + f].x;
                        acc.y += wgt * v[e * 4 + f].y;
                    }
            }
            bc[lt] = acc;
        }
    };
    auto prolong = [&](int k, unsigned xoff) {             // x_k += P x_{k+1} on own fine points
        const SmLevel& L = a.lv[k];
        const SmLevel& Lc = a.lv[k + 1];
        const int own = nown(L);
        V* x = vec(xoff);
        for (int lt = tid; lt < own; lt += nth) {
            int j, i;
            own_rc(L, lt, j, i);
            if (!valid_pt(type, i, j)) continue;
            float px[3], pz[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                px[e] = pw_axis_t<float>(nodx, L.n1, i, (i >> 1) - 1 + e);
                pz[e] = pw_axis_t<float>(nodz, L.n2, j, (j >> 1) - 1 + e);
            }
            V v[9];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const bool rok = pz[e] != 0.f;
                const uint32_t ra = row_addr(Lc, Lc.off_x, rok ? (j >> 1) - 1 + e : 0);
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const bool ok = rok && px[f] != 0.f;
                    v[e * 3 + f] = ld_cluster_at(ra + (uint32_t)(ok ? (i >> 1) - 1 + f : 0) * 8u);
                }
            }
            V acc = x[lt];
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float wgt = pz[e] * px[f];
                    acc.x += wgt * v[e * 3 + f].x;
                    acc.y += wgt * v[e * 3 + f].y;
                }
            x[lt] = acc;
        }
    };
    auto coarse = [&]() {                                   // x_c = A_c^{-1} b_c on own rows, in FP64
        const SmLevel& L = a.lv[kc];
        const int npc = L.n1 * L.n2, own = nown(L), g0 = p0(L);
        V* gath = vec(a.off_g);
        for (int g = tid; g < npc; g += nth) gath[g] = ld_cluster_at(row_addr(L, L.off_b, g / L.n1) + (uint32_t)(g % L.n1) * 8u);
        __syncthreads();
        V* x = vec(L.off_x);
        const int lane = tid & 31;
        for (int row = tid >> 5; row < own; row += nth >> 5) {
            // the FP64 inverse row from global memory (L2-resident), eight loads in flight per lane
            const double2* arow = a.inv[z] + (size_t)(g0 + row) * npc;
            double re = 0.0, im = 0.0;
            auto mac = [&](const double2& m, const V& v) {
                const double vx = (double)v.x, vy = (double)v.y;
                re = fma(m.x, vx, re);
                re = fma(-m.y, vy, re);
                im = fma(m.x, vy, im);
                im = fma(m.y, vx, im);
            };
            int c = lane;
            for (; c + 32 * 7 < npc; c += 32 * 8) {
                double2 m[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) m[u] = __ldg(arow + c + 32 * u);
#pragma unroll
                for (int u = 0; u < 8; ++u) mac(m[u], gath[c + 32 * u]);
            }
            for (; c < npc; c += 32) mac(__ldg(arow + c), gath[c]);
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == 0) x[row] = cmk<V>((float)re, (float)im);
        }
    };
    auto zero_vec = [&](int k, unsigned off) {
        V* x = vec(off);
        for (int lt = tid; lt < nown(a.lv[k]); lt += nth) x[lt] = czero<V>();
    };
    auto copy_vec = [&](int k, unsigned from, unsigned to) {
        const V* s = vec(from);
        V* d = vec(to);
        for (int lt = tid; lt < nown(a.lv[k]); lt += nth) d[lt] = s[lt];
    };

    // ---- the cycle: an explicit walk over the recursion of Algorithm 1 ----
    // Each pass of the loop picks the next phase from the per-level state and
    // runs it through one switch, so every phase's code exists once in the
    // kernel (fewer instructions to fetch after other kernels ran on the SM).
    enum { kJacobi, kZero, kResidual, kRestrict, kCoarse, kProlong, kCopy };
    unsigned xs[kMaxLevels], ts[kMaxLevels];
    int pc[kMaxLevels], nsw[kMaxLevels];
    bool warm[kMaxLevels];
    int k = 0;
    pc[0] = 0;
    warm[0] = a.warm != 0;
    while (true) {
        int op = -1, kk = k;
        unsigned u = 0, v = 0;
        bool zero = false;
        if (k == kc) {
            op = kCoarse;
            --k;
        } else {
            const SmLevel& L = a.lv[k];
            switch (pc[k]) {
            case 0: {                                       // entering the visit
                unsigned x = L.off_x, t = L.off_t;
                nsw[k] = 0;
                if (!warm[k]) {
                    // with a zero initial guess, start in the buffer from which the visit's
                    // buffer swaps (the pre-sweeps after the first, and the post-sweeps)
                    // end in off_x, where the parent level and the final store read the
                    // result: no copy phase
                    if (((a.nu_pre >= 1 ? a.nu_pre - 1 : 0) + a.nu_post) & 1) {
                        x = L.off_t;
                        t = L.off_x;
                    }
                    if (a.nu_pre >= 1) {
                        op = kJacobi;
                        zero = true;
                        v = x;
                        nsw[k] = 1;
                    } else {
                        op = kZero;
                        u = x;
                    }
                }
                xs[k] = x;
                ts[k] = t;
                pc[k] = 1;
                break;
            }
            case 1:                                         // pre-sweeps, then the residual
                if (nsw[k] < a.nu_pre) {
                    op = kJacobi;
                    u = xs[k];
                    v = ts[k];
                    ts[k] = u;
                    xs[k] = v;
                    ++nsw[k];
                } else {
                    op = kResidual;
                    u = xs[k];
                    v = ts[k];
                    pc[k] = 2;
                }
                break;
            case 2:
                op = kRestrict;
                u = ts[k];
                pc[k] = 3;
                break;
            case 3:                                         // the coarse visit(s)
                pc[k] = (a.wcycle && k + 1 < kc) ? 4 : 5;
                ++k;
                pc[k] = 0;
                warm[k] = false;
                break;
            case 4:                                         // the W-cycle's second coarse visit
                pc[k] = 5;
                ++k;
                pc[k] = 0;
                warm[k] = true;
                break;
            case 5:
                op = kProlong;
                u = xs[k];
                nsw[k] = 0;
                pc[k] = 6;
                break;
            case 6:                                         // post-sweeps, then the copy to off_x
                if (nsw[k] < a.nu_post) {
                    op = kJacobi;
                    u = xs[k];
                    v = ts[k];
                    ts[k] = u;
                    xs[k] = v;
                    ++nsw[k];
                    break;
                }
                pc[k] = 7;
                if (xs[k] != L.off_x) {
                    op = kCopy;
                    u = xs[k];
                    v = L.off_x;
                    xs[k] = L.off_x;
                }
                break;
            default:                                        // visit done
                break;
            }
            if (op < 0 && pc[kk] == 7) {
                if (kk == 0) break;
                k = kk - 1;
            }
        }
        if (op < 0) continue;
        switch (op) {
        case kJacobi: jacobi(kk, u, v, zero); break;
        case kZero: zero_vec(kk, u); break;
        case kResidual: residual(kk, u, v); break;
        case kRestrict: restrict_(kk, u); break;
        case kCoarse: coarse(); break;
        case kProlong: prolong(kk, u); break;
        default: copy_vec(kk, u, v); break;
        }
        cluster_barrier();
    }

    // ---- store the level-l0 result; keep shared memory alive for remote readers ----
    {
        const SmLevel& L = a.lv[0];
        const int own = nown(L), g0 = p0(L);
        const size_t roff = (size_t)rr * L.n1 * L.n2 + g0;
        const V* x = vec(L.off_x);
        for (int t = tid; t < own; t += nth) a.gx[z][roff + t] = x[t];
    }
    cluster_barrier();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static const void* smmg_fn(int rm) {
    return rm <= 1 ? (const void*)k_cluster_mg<1> : (const void*)k_cluster_mg<2>;
}

size_t smmg_layout(SmArgs& a, const int* n1, const int* n2, const int* nslot_max, int nlev, int cs) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 15) & ~size_t(15);
        return (unsigned)o;
    };
    a.nlev = nlev;
    for (int k = 0; k < nlev; ++k) {
        SmLevel& L = a.lv[k];
        L.n1 = n1[k];
        L.n2 = n2[k];
        L.rp = (n2[k] + cs - 1) / cs;
        L.inv_rp = 1.0f / (float)L.rp;
        L.inv_n1 = 1.0f / (float)L.n1;
        const size_t cap = (size_t)L.rp * L.n1;
        if (k < nlev - 1) {
            L.off_c = take(cap * nslot_max[k] * 4);
            L.off_t = take(cap * 8);
        } else {
            L.off_c = 0;
            L.off_t = 0;
        }
        L.off_x = take(cap * 8);
        L.off_b = take(cap * 8);
    }
    const SmLevel& Lc = a.lv[nlev - 1];
    const size_t npc = (size_t)Lc.n1 * Lc.n2;
    a.off_g = take(npc * 8);
    return off;
}

int smmg_prepare(int rm, int cs, size_t smem) {
    const void* fn = smmg_fn(rm);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (cs > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int launch_cluster_mg(const SmArgs& a, int rm, int nrhs, int cs, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * a.nb * nrhs);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e = rm <= 1 ? cudaLaunchKernelEx(&cfg, k_cluster_mg<1>, a) : cudaLaunchKernelEx(&cfg, k_cluster_mg<2>, a);
    return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace bah
