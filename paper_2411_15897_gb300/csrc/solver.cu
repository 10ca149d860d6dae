// Host side of libbah: context construction, the multigrid cycle schedule,
// the block-acoustic preconditioner, flexible GMRES, and the C ABI of bah.h.
//
// The preconditioning step (Sec. 3, Eq. 3.1-3.5) is
//     t_p = B v_u - A_p v_p;   e_p = cycle(H_p,s, t_p);
//     s_u = v_u - B^T e_p;     e_u = cycle(A_s, s_u)   (the d blocks in one batch)
// and FGMRES (right preconditioned, two-pass classical Gram-Schmidt, Givens
// rotations on the device) wraps it with the FP64 operator H of Eq. 2.6.
#include "bah_internal.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <utility>

namespace bah {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

#define TRY(expr)                                  \
    do {                                           \
        int _s = (expr);                           \
        if (_s != BAH_OK) return _s;               \
    } while (0)

static const double kAlphaByLevels[5] = {0.0, 0.0, 0.1, 0.2, 0.4};
// deeper hierarchies than the paper's tables: the shift minimising the
// iteration count on the layered and random-field workloads (5-7 levels),
// searched at a resolution of 0.1 as the paper searches its shifts
static const double kAlphaDeep = 1.0;
static const int kIntSlots = 8;

struct Ctx {
    int dim = 2, n1 = 0, n2 = 0, np = 0;
    double h1 = 0, h2 = 0, omega = 0, alpha = 0;
    bah_opts o{};
    int L = 1;
    int mode = BAH_MIXED;
    size_t vsz = 8;                      // bytes of one complex entry in the preconditioner's precision
    std::vector<void*> allocs;

    // FP64 coefficient arrays (cells)
    double *cx = nullptr, *cz = nullptr, *nx = nullptr, *nz = nullptr, *wx = nullptr, *wz = nullptr, *cinv = nullptr;
    double2 *d1 = nullptr, *d2 = nullptr, *dg[3] = {nullptr, nullptr, nullptr}, *dAp = nullptr;
    double* gam = nullptr;               // attenuation at cells (device), for the gradient
    OpCoef op{};
    OpCoefDF opdf{};                     // double-float copies (mixed mode with the double-float basis)
    bool opdf_ok = false;
    // level-0 arrays in storage precision
    void *s_cx = nullptr, *s_cz = nullptr, *s_nx = nullptr, *s_nz = nullptr, *s_wx = nullptr, *s_wz = nullptr;
    void *s_dg[3] = {nullptr, nullptr, nullptr}, *s_dAp = nullptr;
    // hierarchy
    std::vector<int> ln1, ln2;
    std::vector<std::array<StencilF64, 3>> s64;   // FP64 stencils per level (level 0: 3x3 fine operator)
    std::vector<std::array<void*, 3>> sst;        // storage-precision stencils, levels >= 1
    double2* inv[3] = {nullptr, nullptr, nullptr};
    std::vector<std::array<void*, 3>> vX, vB, vT; // multigrid vectors per level and block
    // Krylov workspace
    int m = 20;
    double2 *V = nullptr, *W = nullptr, *R = nullptr, *Bs = nullptr, *X = nullptr;
    double2 *Hm = nullptr, *h1v = nullptr, *h2v = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double2* partial = nullptr;
    double *nrm = nullptr, *dpart = nullptr, *status = nullptr;
    void* Z = nullptr;
    double* hstatus = nullptr;           // pinned host mirror of status
    void* ztmp = nullptr;                // preconditioner output in storage precision (apply hook)
    // right-hand-side batching
    int nbatch = 1;                      // right-hand sides solved together
    bool kdf = false;                    // Krylov basis in double-float (BAH_KRYLOV_DF)
    int* active = nullptr;               // device, per right-hand side
    int* jk = nullptr;                   // device, Krylov dimension per right-hand side at a restart
    int* hint = nullptr;                 // pinned host staging ring for active / jk (kIntSlots * nbatch)
    unsigned hint_slot = 0;
    KS ks;                               // strides of the batched Krylov workspace

    // profiling: launch counts, algorithmic bytes, event timing per kernel class
    unsigned tmask = 0;
    long long launches = 0;
    long long cls_launch[16] = {}, cls_calls[16] = {};
    double cls_ms[16] = {}, cls_bytes[16] = {};
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    std::vector<std::pair<int, size_t>> pending;

    // Gram-Schmidt flag and per-step graphs
    int* gsflag = nullptr;
    struct IterGraph {
        cudaGraphExec_t exec = nullptr;
        unsigned mask = ~0u;
        long long launches = 0, cls_launch[16] = {}, cls_calls[16] = {};
        double cls_bytes[16] = {};
        std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    };
    std::vector<IterGraph> ig;
    IterGraph* capturing = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaEvent_t> itev;
    bool use_graphs = true;
    bool staged = true;                  // shared-memory staging of Galerkin-level sweeps (BAH_STAGED=0: off)
    double dgks_eta2 = 0.5;              // second Gram-Schmidt pass when ||w'||^2 < eta2 ||w||^2
    int sm_l0 = 0;                       // first level of the shared-memory cluster multigrid (0: off)
    int sm_cs = 0, sm_rm = 2;            // its CTAs per cluster and stencil radius bound
    size_t sm_bytes = 0;                 // its dynamic shared memory per CTA
    int nsm = 0;

    // exact-block preconditioner (block_rtol > 0): each acoustic block solved
    // by an inner FGMRES(mi) in FP64, preconditioned by its multigrid cycle
    bool exact = false;
    Fine5<double, double2> f5x{};       // FP64 block operators, diagonals shifted by block_alpha
    int mi = 60;                        // inner restart length
    double2 *iV = nullptr, *iZ = nullptr, *iW = nullptr, *iR = nullptr, *iH = nullptr;
    double2 *ih1 = nullptr, *ih2 = nullptr, *ics = nullptr, *isn = nullptr, *igv = nullptr, *iy = nullptr;
    double2* ipart = nullptr;
    double *inrm = nullptr, *idpart = nullptr, *istatus = nullptr;
    int *iflag = nullptr, *ijk = nullptr;
    double* histat = nullptr;           // pinned: 8 status / norm slots and one int
    double2 *ez = nullptr, *etp = nullptr, *esu = nullptr;
    long long block_iters = 0;
    int block_failures = 0;
    int exact_status = BAH_OK;          // first failure of a block solve inside a preconditioner call

    // block FGMRES workspace (block_krylov = 1)
    double2 *bC = nullptr, *bT = nullptr, *bpart = nullptr;
    double2* bhost = nullptr;           // pinned

    // three-dimensional grids (dim == 3): n1 x n2 x n3 cells
    int n3 = 1;
    double h3 = 0;
    Op3 op3{};
    std::vector<std::array<int, 3>> d3;            // level grids
    std::vector<std::array<double2*, 4>> s3;       // FP64 stencils (level 0: 7-point, coarser: 27-point)
    std::vector<std::array<void*, 4>> s3s;         // the same in storage precision, bf16 in mixed mode (levels below the coarsest)
    std::vector<std::array<void*, 4>> v3B, v3X, v3T;
    double2* inv3[4] = {nullptr, nullptr, nullptr, nullptr};

    static void clear_graph(IterGraph& G) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        for (auto& e : G.ev) { cudaEventDestroy(e.second.first); cudaEventDestroy(e.second.second); }
        G = IterGraph();
    }

    ~Ctx() {
        for (auto& G : ig) clear_graph(G);
        for (cudaEvent_t e : itev) cudaEventDestroy(e);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (cudaEvent_t e : evpool) cudaEventDestroy(e);
        for (void* p : allocs) cudaFree(p);
        if (hstatus) cudaFreeHost(hstatus);
        if (hint) cudaFreeHost(hint);
        if (histat) cudaFreeHost(histat);
        if (bhost) cudaFreeHost(bhost);
    }
    int alloc(void** p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
            return BAH_ERR_OOM;
        }
        allocs.push_back(*p);
        return BAH_OK;
    }
    template <class T> int alloc_t(T** p, size_t count) {
        void* q;
        int s = alloc(&q, count * sizeof(T));
        *p = (T*)q;
        return s;
    }
    size_t vec_len() const { return (size_t)(dim + 1) * np; }
};

// ---------------------------------------------------------------------------
// profiling scope: counts the kernels of one launcher call and its algorithmic
// bytes; for timed classes brackets the launch with events on its stream
// ---------------------------------------------------------------------------
static void prof_flush(Ctx& c) {
    if (c.pending.empty()) return;
    cudaEventSynchronize(c.evpool[c.pending.back().second + 1]);
    for (auto& pr : c.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.evpool[pr.second], c.evpool[pr.second + 1]) == cudaSuccess)
            c.cls_ms[pr.first] += ms;
    }
    cudaGetLastError();
    c.pending.clear();
    c.evused = 0;
}

struct Prof {
    Ctx& c;
    int cls;
    cudaStream_t st;
    double bytes;
    int nk;
    size_t idx = (size_t)-1;
    cudaEvent_t ce0 = nullptr, ce1 = nullptr;
    Prof(Ctx& c_, int cls_, cudaStream_t st_, double bytes_, int nk_ = 1)
        : c(c_), cls(cls_), st(st_), bytes(bytes_), nk(nk_) {
        if (c.capturing) {
            if (c.tmask & (1u << cls)) {
                if (cudaEventCreate(&ce0) == cudaSuccess && cudaEventCreate(&ce1) == cudaSuccess) {
                    // an external record becomes an event-record node of the graph, replayed per launch
                    cudaEventRecordWithFlags(ce0, st, cudaEventRecordExternal);
                } else {
                    cudaGetLastError();
                    ce0 = ce1 = nullptr;
                }
            }
            return;
        }
        if (c.tmask & (1u << cls)) {
            if (c.evused + 2 > c.evpool.size()) {
                if (c.evpool.size() < 16384) {
                    for (int k = 0; k < 2; ++k) {
                        cudaEvent_t e;
                        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
                        c.evpool.push_back(e);
                    }
                } else {
                    prof_flush(c);
                }
            }
            idx = c.evused;
            c.evused += 2;
            cudaEventRecord(c.evpool[idx], st);
        }
    }
    ~Prof() {
        if (c.capturing) {
            auto* G = c.capturing;
            if (ce0) {
                cudaEventRecordWithFlags(ce1, st, cudaEventRecordExternal);
                G->ev.push_back({cls, {ce0, ce1}});
            }
            G->launches += nk;
            G->cls_launch[cls] += nk;
            G->cls_calls[cls] += 1;
            G->cls_bytes[cls] += bytes;
            return;
        }
        if (idx != (size_t)-1) {
            cudaEventRecord(c.evpool[idx + 1], st);
            c.pending.emplace_back(cls, idx);
        }
        c.launches += nk;
        c.cls_launch[cls] += nk;
        c.cls_calls[cls] += 1;
        c.cls_bytes[cls] += bytes;
    }
};

// right-hand sides of one launch and their active flags
struct Batch {
    int nr = 1;
    const int* active = nullptr;
};

// ---------------------------------------------------------------------------
// multigrid cycle over a set of blocks (Algorithm 1 applied recursively)
// ---------------------------------------------------------------------------
template <int MODE>
struct MG {
    using V = typename Prec<MODE>::V;
    using C = typename Prec<MODE>::C;
    using CC = typename Prec<MODE>::CC;

    static Fine5<C, CC> fine5(const Ctx& c) {
        Fine5<C, CC> f;
        f.n1 = c.n1; f.n2 = c.n2;
        f.cx = (const C*)c.s_cx; f.cz = (const C*)c.s_cz; f.nx = (const C*)c.s_nx; f.nz = (const C*)c.s_nz;
        f.wx = (const C*)c.s_wx; f.wz = (const C*)c.s_wz;
        f.dg0 = (const CC*)c.s_dg[0]; f.dg1 = (const CC*)c.s_dg[1]; f.dg2 = (const CC*)c.s_dg[2];
        f.dAp = (const CC*)c.s_dAp;
        return f;
    }

    static double weight(const Ctx& c, int l) {
        int k = std::min(l, c.o.n_jacobi_w - 1);
        return c.o.jacobi_w[k];
    }

    static LvlSet<V, CC> set(const Ctx& c, int l, int b0, int nb, V* const* xin, size_t sxi, V* const* xout,
                             size_t sxo, const Batch& bt) {
        LvlSet<V, CC> s;
        std::memset(&s, 0, sizeof(s));
        s.nb = nb; s.n1 = c.ln1[l]; s.n2 = c.ln2[l];
        s.nrhs = bt.nr;
        s.active = bt.active;
        s.staged = c.staged ? 1 : 0;
        const size_t npl = (size_t)c.ln1[l] * c.ln2[l];
        for (int z = 0; z < nb; ++z) {
            const int b = b0 + z;
            auto& B = s.blk[z];
            B.type = b;
            B.S = l > 0 ? (const CC*)c.sst[l][b] : nullptr;
            B.rx = c.s64[l][b].rx; B.rz = c.s64[l][b].rz;
            B.b = (const V*)c.vB[l][b];
            B.sb = npl;
            B.xin = xin ? xin[z] : nullptr;
            B.sxi = sxi;
            B.xout = xout[z];
            B.sxo = sxo;
        }
        return s;
    }

    // algorithmic bytes of one sweep-type launch on level l for blocks [b0, b0+nb)
    static double coef_bytes(const Ctx& c, int l, int b0, int nb) {
        const double cs = sizeof(C), ccs = sizeof(CC);
        const double npl = (double)c.ln1[l] * c.ln2[l];
        double t = 0;
        for (int b = b0; b < b0 + nb; ++b) {
            if (l == 0) t += npl * (((b == 2 && c.h1 == c.h2) ? 1.0 : 2.0) * cs + ccs);
            else t += npl * ccs * (2 * c.s64[l][b].rx + 1) * (2 * c.s64[l][b].rz + 1);
        }
        return t;
    }

    // levels sm_l0..L-1 held in one cluster's shared memory per block and
    // right-hand side (mixed mode): right-hand sides in vB[sm_l0], results in
    // vX[sm_l0]; warm: start from the values in vX[sm_l0]
    static void smem_levels(Ctx& c, int b0, int nb, const Batch& bt, cudaStream_t st, bool warm = false) {
        if constexpr (MODE == BAH_MIXED) {
            SmArgs a;
            std::memset(&a, 0, sizeof(a));
            const int l0 = c.sm_l0, nlev = c.L - l0;
            int n1s[kMaxLevels], n2s[kMaxLevels], ns[kMaxLevels];
            for (int k = 0; k < nlev; ++k) {
                n1s[k] = c.ln1[l0 + k]; n2s[k] = c.ln2[l0 + k];
                ns[k] = 0;
                for (int b = 0; b < 3; ++b)
                    ns[k] = std::max(ns[k], (2 * c.s64[l0 + k][b].rx + 1) * (2 * c.s64[l0 + k][b].rz + 1));
            }
            smmg_layout(a, n1s, n2s, ns, nlev, c.sm_cs);
            for (int k = 0; k < nlev; ++k) a.lv[k].w = (float)weight(c, l0 + k);
            a.b0 = b0; a.nb = nb; a.nu_pre = c.o.nu_pre; a.nu_post = c.o.nu_post; a.intergrid = c.o.intergrid;
            a.wcycle = c.o.cycle == BAH_CYCLE_W; a.warm = warm; a.active = bt.active;
            for (int z = 0; z < nb; ++z) {
                const int b = b0 + z;
                for (int k = 0; k < nlev - 1; ++k) {
                    a.S[z][k] = (const __nv_bfloat162*)c.sst[l0 + k][b];
                    a.rx[z][k] = c.s64[l0 + k][b].rx; a.rz[z][k] = c.s64[l0 + k][b].rz;
                }
                a.gb[z] = (const float2*)c.vB[l0][b];
                a.gx[z] = (float2*)c.vX[l0][b];
                a.inv[z] = c.inv[b];
            }
            double bytes = 0;
            for (int k = 0; k < nlev - 1; ++k) bytes += coef_bytes(c, l0 + k, b0, nb) * bt.nr;
            const double npc = (double)c.ln1[c.L - 1] * c.ln2[c.L - 1];
            bytes += nb * bt.nr * (npc * npc * 16.0 + (double)c.ln1[l0] * c.ln2[l0] * 8.0 * (warm ? 3 : 2));
            Prof pr(c, BAH_K_CLUSTER, st, bytes);
            launch_cluster_mg(a, c.sm_rm, bt.nr, c.sm_cs, c.sm_bytes, st);
        }
    }

    // One cycle on level l for blocks [b0, b0+nb) and bt.nr right-hand sides:
    // right-hand sides in vB[l][b] (stride npl), results written to out[z] with
    // right-hand-side stride ostride.  The initial guess is zero, or (x0) the
    // values already in out[z].  A W-cycle visits the coarse problem twice: the
    // second visit starts from the first one's result (Sec. 2.2, two recursive
    // calls), except when the coarse level is the coarsest, solved exactly once.
    static void cycle(Ctx& c, int l, int b0, int nb, V* const* out, size_t ostride, const Batch& bt,
                      cudaStream_t st, bool x0 = false) {
        const size_t npl = (size_t)c.ln1[l] * c.ln2[l];
        const double vs = sizeof(V), ccs = sizeof(CC);
        const double nr = bt.nr;
        if (l == c.L - 1) {
            const double2* inv[3];
            const V* bb[3];
            V* xx[3];
            for (int z = 0; z < nb; ++z) { inv[z] = c.inv[b0 + z]; bb[z] = (const V*)c.vB[l][b0 + z]; xx[z] = out[z]; }
            RhsStride rs;
            rs.s0 = npl; rs.s1 = ostride; rs.active = bt.active;
            Prof pr(c, BAH_K_COARSE, st, nb * (double)npl * npl * 16.0 + nr * nb * 2.0 * npl * vs);
            launch_coarse_apply<MODE>(nb, (int)npl, inv, bb, xx, st, bt.nr, rs);
            return;
        }
        Fine5<C, CC> f5 = fine5(c);
        const Fine5<C, CC>* pf5 = l == 0 ? &f5 : nullptr;
        const double w = weight(c, l);
        const double cb_ = coef_bytes(c, l, b0, nb);
        const double sweep = cb_ + 3.0 * vs * npl * nb * nr;
        const size_t nplc = npl / 4;
        V* cur[3];
        V* oth[3];
        size_t cur_s = ostride, oth_s = npl;
        for (int z = 0; z < nb; ++z) { cur[z] = out[z]; oth[z] = (V*)c.vT[l][b0 + z]; }
        auto swap_cur = [&]() {
            for (int z = 0; z < nb; ++z) std::swap(cur[z], oth[z]);
            std::swap(cur_s, oth_s);
        };
        V* cb[3];
        V* cx[3];
        for (int z = 0; z < nb; ++z) { cb[z] = (V*)c.vB[l + 1][b0 + z]; cx[z] = (V*)c.vX[l + 1][b0 + z]; }
        const bool wcyc = c.o.cycle == BAH_CYCLE_W;
        {
            // With a zero initial guess the caller's buffer holds nothing yet: if the
            // sweeps below swap the two buffers an odd number of times, start in the
            // other one, so that the last sweep lands in the caller's buffer and no
            // copy is needed.
            if (!x0 && ((std::max(c.o.nu_pre - 1, 0) + c.o.nu_post) & 1)) swap_cur();
            // pre-relaxation
            if (x0) {
                for (int s = 0; s < c.o.nu_pre; ++s) {
                    Prof pr(c, BAH_K_JACOBI, st, sweep);
                    launch_jacobi<MODE>(set(c, l, b0, nb, cur, cur_s, oth, oth_s, bt), pf5, w, 0, st);
                    swap_cur();
                }
            } else if (c.o.nu_pre >= 1) {
                {
                    Prof pr(c, BAH_K_JACOBI, st, nr * nb * npl * (2.0 * vs + ccs));
                    launch_jacobi<MODE>(set(c, l, b0, nb, nullptr, 0, cur, cur_s, bt), pf5, w, 1, st);
                }
                for (int s = 1; s < c.o.nu_pre; ++s) {
                    Prof pr(c, BAH_K_JACOBI, st, sweep);
                    launch_jacobi<MODE>(set(c, l, b0, nb, cur, cur_s, oth, oth_s, bt), pf5, w, 0, st);
                    swap_cur();
                }
            } else {
                Prof pr(c, BAH_K_SMALL, st, nr * nb * npl * vs, 0);
                for (int z = 0; z < nb; ++z)
                    cudaMemset2DAsync(cur[z], cur_s * sizeof(V), 0, npl * sizeof(V), bt.nr, st);
            }
            // residual and restriction
            auto rs = set(c, l, b0, nb, cur, cur_s, oth, oth_s, bt);
            {
                Prof pr(c, BAH_K_RESIDUAL, st, sweep);
                launch_residual<MODE>(rs, pf5, st);
            }
            {
                Prof pr(c, BAH_K_RESTRICT, st, nr * nb * npl * vs * 1.25);
                launch_restrict<MODE>(rs, cb, c.o.intergrid, st, nplc);
            }
            // coarse-grid correction
            if (c.sm_l0 == l + 1) {
                smem_levels(c, b0, nb, bt, st);
                if (wcyc && l + 1 < c.L - 1) smem_levels(c, b0, nb, bt, st, true);
            } else {
                cycle(c, l + 1, b0, nb, cx, nplc, bt, st);
                if (wcyc && l + 1 < c.L - 1) cycle(c, l + 1, b0, nb, cx, nplc, bt, st, true);
            }
            {
                Prof pr(c, BAH_K_PROLONG, st, nr * nb * npl * vs * 2.25);
                launch_prolong_add<MODE>(set(c, l, b0, nb, nullptr, 0, cur, cur_s, bt), cx, st, nplc);
            }
            // post-relaxation
            for (int s = 0; s < c.o.nu_post; ++s) {
                Prof pr(c, BAH_K_JACOBI, st, sweep);
                launch_jacobi<MODE>(set(c, l, b0, nb, cur, cur_s, oth, oth_s, bt), pf5, w, 0, st);
                swap_cur();
            }
        }
        for (int z = 0; z < nb; ++z)
            if (cur[z] != out[z]) {
                Prof pr(c, BAH_K_SMALL, st, 2.0 * nr * npl * vs, 0);
                cudaMemcpy2DAsync(out[z], ostride * sizeof(V), cur[z], cur_s * sizeof(V), npl * sizeof(V), bt.nr,
                                  cudaMemcpyDeviceToDevice, st);
            }
    }

    // z = P^{-1} D r for bt.nr right-hand sides  (r FP64 padded vectors with
    // stride rs, z storage-precision padded vectors with stride zs)
    template <class RIN>
    static void precond(Ctx& c, const RIN* r, size_t rstride, V* z, size_t zstride, const Batch& bt,
                        cudaStream_t st) {
        const int np = c.np;
        const double vs = sizeof(V);
        Fine5<C, CC> f5 = fine5(c);
        {
            RhsStride rs;
            rs.s0 = rstride; rs.s1 = np; rs.active = bt.active;
            Prof pr(c, BAH_K_DISTRIB, st, (double)bt.nr * np * (48.0 + sizeof(C) + sizeof(CC) + vs));
            launch_distributor<MODE, RIN>(c.n1, c.n2, 1.0 / c.h1, 1.0 / c.h2, f5, r, (V*)c.vB[0][2], st, bt.nr, rs);
        }
        V* outp[1] = {z + 2 * (size_t)np};
        cycle(c, 0, 2, 1, outp, zstride, bt, st);
        {
            RhsStride rs;
            rs.s0 = rstride; rs.s1 = zstride; rs.s2 = np; rs.active = bt.active;
            Prof pr(c, BAH_K_URHS, st, (double)bt.nr * np * (32.0 + 3.0 * vs));
            launch_u_rhs<MODE, RIN>(c.n1, c.n2, 1.0 / c.h1, 1.0 / c.h2, r, z + 2 * (size_t)np, (V*)c.vB[0][0],
                                    (V*)c.vB[0][1], st, bt.nr, rs);
        }
        V* outu[2] = {z, z + (size_t)np};
        cycle(c, 0, 0, 2, outu, zstride, bt, st);
    }
};

// ---------------------------------------------------------------------------
// three-dimensional multigrid: the cycle of one block, or of the three
// displacement blocks in the same launches (Algorithm 1 applied recursively; a
// W-cycle visits every level below the first twice, the second visit starting
// from the first's result) and the block-acoustic preconditioner
// e = P^{-1} D r (Eq. 3.3 - 3.5) with its four blocks
// ---------------------------------------------------------------------------
template <int MODE>
struct MG3 {
    using V = typename Prec<MODE>::V;
    static size_t pts(const Ctx& c, int l) { return (size_t)c.d3[l][0] * c.d3[l][1] * c.d3[l][2]; }
    static double jw(const Ctx& c, int l) { return c.o.jacobi_w[std::min(l, c.o.n_jacobi_w - 1)]; }
    // for blocks q0 .. q0 + nq - 1 of level l in one launch: x_out = Jacobi sweep
    // from x_in (zero: from x_in = 0), or x_out = b - A x_in (res)
    static void sweep(Ctx& c, int l, int q0, int nq, V* const* xin, V* const* xout, int zero, int res,
                      cudaStream_t st) {
        const int ns = l == 0 ? 7 : 27;
        const double vb = sizeof(V);
        const double sb = MODE == BAH_MIXED ? 4.0 : 16.0;          // bytes per stored stencil entry
        Prof pr(c, res ? BAH_K_RESIDUAL : BAH_K_JACOBI, st, (double)nq * pts(c, l) * (ns * sb + (zero ? 2.0 : 3.0) * vb));
        const void* S[3];
        const V* b[3];
        const V* xi[3];
        for (int y = 0; y < nq; ++y) {
            S[y] = c.s3s[l][q0 + y];
            b[y] = (const V*)c.v3B[l][q0 + y];
            xi[y] = xin[y];
        }
        launch_jacobi3<V>(q0, nq, c.d3[l].data(), ns, S, b, xi, xout, jw(c, l), zero, res, st);
    }
    // x_y = approximately A_{q0+y}^{-1} b_{q0+y} on level l for y < nq (b in v3B[l]),
    // all blocks in the same launches; zero: zero initial guess, else start from x
    static void cycle(Ctx& c, int l, int q0, int nq, V* const* x, bool zero, cudaStream_t st) {
        const size_t np = pts(c, l);
        if (l == c.L - 1) {
            const double vb = sizeof(V);
            Prof pr(c, BAH_K_COARSE, st, nq * ((double)np * np * 16.0 + 2.0 * np * vb));
            const double2* inv[3];
            const V* bb[3];
            for (int y = 0; y < nq; ++y) {
                inv[y] = c.inv3[q0 + y];
                bb[y] = (const V*)c.v3B[l][q0 + y];
            }
            launch_coarse_apply<MODE>(nq, (int)np, inv, bb, x, st);
            return;
        }
        // the two buffers of each block's ping-pong; the current iterate is in A[y] when inA
        V* A[3] = {nullptr, nullptr, nullptr};
        V* B[3] = {nullptr, nullptr, nullptr};
        for (int y = 0; y < nq; ++y) {
            A[y] = x[y];
            B[y] = (V*)c.v3T[l][q0 + y];
        }
        bool inA = true;
        auto cur = [&]() { return inA ? A : B; };
        auto spare = [&]() { return inA ? B : A; };
        int s0 = 0;
        if (zero) {
            s0 = c.o.nu_pre >= 1 ? 1 : 0;
            // start the ping-pong so that the last sweep writes x
            if (((c.o.nu_pre - s0) + c.o.nu_post) % 2) inA = false;
            if (s0) sweep(c, l, q0, nq, cur(), cur(), 1, 0, st);
            else
                for (int y = 0; y < nq; ++y) cudaMemsetAsync(cur()[y], 0, np * sizeof(V), st);
        }
        for (int s = s0; s < c.o.nu_pre; ++s) {
            sweep(c, l, q0, nq, cur(), spare(), 0, 0, st);
            inA = !inA;
        }
        sweep(c, l, q0, nq, cur(), spare(), 0, 1, st);
        V* bc[3] = {nullptr, nullptr, nullptr};
        V* xc[3] = {nullptr, nullptr, nullptr};
        for (int y = 0; y < nq; ++y) {
            bc[y] = (V*)c.v3B[l + 1][q0 + y];
            xc[y] = (V*)c.v3X[l + 1][q0 + y];
        }
        {
            Prof pr(c, BAH_K_RESTRICT, st, nq * (double)np * sizeof(V) * 1.125);
            const V* r[3] = {spare()[0], spare()[1], spare()[2]};
            launch_restrict3<V>(q0, nq, c.d3[l].data(), r, bc, st);
        }
        cycle(c, l + 1, q0, nq, xc, true, st);
        if (c.o.cycle == BAH_CYCLE_W && l + 1 < c.L - 1) cycle(c, l + 1, q0, nq, xc, false, st);
        {
            Prof pr(c, BAH_K_PROLONG, st, nq * (double)np * sizeof(V) * 2.125);
            const V* e[3] = {xc[0], xc[1], xc[2]};
            launch_prolong3<V>(q0, nq, c.d3[l].data(), e, cur(), st);
        }
        for (int s = 0; s < c.o.nu_post; ++s) {
            sweep(c, l, q0, nq, cur(), spare(), 0, 0, st);
            inA = !inA;
        }
        if (!inA)
            for (int y = 0; y < nq; ++y) cudaMemcpyAsync(x[y], B[y], np * sizeof(V), cudaMemcpyDeviceToDevice, st);
    }
    // z = P^{-1} D r for one right-hand side (r FP64, z in the cycle's type):
    // the pressure block's cycle, then the three displacement blocks' cycles
    // together
    static void precond(Ctx& c, const double2* r, V* z, cudaStream_t st) {
        const size_t np = c.np;
        const double vb = sizeof(V);
        {
            Prof pr(c, BAH_K_DISTRIB, st, (double)np * (64.0 + 56.0 + vb));
            launch_distrib3<V>(c.op3, r, (V*)c.v3B[0][3], st);
        }
        V* zp[1] = {z + 3 * np};
        cycle(c, 0, 3, 1, zp, true, st);
        {
            V* su[3] = {(V*)c.v3B[0][0], (V*)c.v3B[0][1], (V*)c.v3B[0][2]};
            Prof pr(c, BAH_K_URHS, st, (double)np * (48.0 + 4.0 * vb));
            launch_urhs3<V>(c.op3, r, z + 3 * np, su, st);
        }
        V* zu[3] = {z, z + np, z + 2 * np};
        cycle(c, 0, 0, 3, zu, true, st);
    }
};

// ---------------------------------------------------------------------------
// exact-block preconditioner (block_rtol > 0; Sec. 4.1, Table 2; Theorem 1):
// every acoustic block is solved, not approximated.  The inner solver is
// FGMRES(mi) in FP64 on the block's fine operator (shifted by block_alpha),
// right preconditioned by the block's multigrid cycle in the context's
// precision; x_0 = 0; it stops when ||s - M e|| <= block_rtol ||s||.  Driven
// from the host (one status read per inner iteration), so these calls are
// not captured in graphs.
// ---------------------------------------------------------------------------
static int read_dev_double(Ctx& c, const double* dev, double* out, cudaStream_t st) {
    BAH_CUDA_TRY(cudaMemcpyAsync(c.histat, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    *out = c.histat[0];
    return BAH_OK;
}

template <int MODE>
static int block_solve(Ctx& c, int b, const double2* s, double2* e, cudaStream_t st) {
    using V = typename Prec<MODE>::V;
    const size_t np = c.np;
    const int m = c.mi;
    const double rtol = c.o.block_rtol;
    KS ks;                                  // one right-hand side: no strides, no flags
    Batch one;
    launch_norm2(s, np, c.idpart, c.inrm, 1, 1, ks, st);
    double bn = 0.0;
    TRY(read_dev_double(c, c.inrm + 1, &bn, st));
    BAH_CUDA_TRY(cudaMemsetAsync(e, 0, np * sizeof(double2), st));
    if (!std::isfinite(bn)) return BAH_ERR_NONFINITE;
    if (!(bn > 0.0)) return BAH_OK;
    BAH_CUDA_TRY(cudaMemcpyAsync(c.iR, s, np * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(c.inrm, c.inrm + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
    double beta = bn;
    int total = 0;
    while (beta > rtol * bn) {
        if (total >= c.o.block_maxit) { ++c.block_failures; break; }
        launch_scale_copy(c.iR, c.inrm, 0, c.iV, np, 0, 0, 1, ks, st);
        launch_init_arnoldi(c.inrm, c.igv, m, c.istatus, 1, ks, st);
        int jd = 0;
        for (int j = 0; j < m && total < c.o.block_maxit; ++j) {
            const double2* vj = c.iV + (size_t)j * np;
            double2* zj = c.iZ + (size_t)j * np;
            // z_j = (one multigrid cycle of the block) v_j
            if constexpr (MODE == BAH_MIXED) {
                launch_convert<double2, float2>(vj, (float2*)c.vB[0][b], np, st);
                V* o[1] = {(V*)c.ztmp};
                MG<MODE>::cycle(c, 0, b, 1, o, np, one, st);
                launch_convert<float2, double2>((const float2*)c.ztmp, zj, np, st);
            } else {
                BAH_CUDA_TRY(cudaMemcpyAsync(c.vB[0][b], vj, np * sizeof(double2), cudaMemcpyDeviceToDevice, st));
                V* o[1] = {zj};
                MG<MODE>::cycle(c, 0, b, 1, o, np, one, st);
            }
            // w = M z_j, Gram-Schmidt with selective reorthogonalisation, Givens, v_{j+1}
            launch_block_apply64(c.f5x, b, zj, c.iW, nullptr, st);
            launch_dot_norm(c.iV, j + 1, c.iW, np, c.ipart, c.ih1, nullptr, 1, ks, st);
            launch_axpy_norm(c.iV, j + 1, c.ih1, c.iW, np, c.idpart, nullptr, 1, ks, st);
            launch_dgks_decide(c.idpart, c.ih1, j + 1, c.iflag, c.inrm, 1, ks, st);
            launch_dot_norm(c.iV, j + 1, c.iW, np, c.ipart, c.ih2, c.iflag, 1, ks, st);
            launch_axpy_norm(c.iV, j + 1, c.ih2, c.iW, np, c.idpart, c.iflag, 1, ks, st);
            launch_pass2_norm(c.idpart, c.iflag, c.inrm, 1, ks, st);
            launch_arnoldi_givens(c.iH, m + 1, c.ih1, c.ih2, c.inrm, j, c.ics, c.isn, c.igv, c.istatus, 1, ks, st);
            launch_scale_copy(c.iW, c.inrm, 2, c.iV + (size_t)(j + 1) * np, np, 0, 0, 1, ks, st);
            BAH_CUDA_TRY(cudaMemcpyAsync(c.histat, c.istatus, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            BAH_CUDA_TRY(cudaStreamSynchronize(st));
            ++total;
            jd = j + 1;
            const double est = c.histat[0] / bn;
            if (c.histat[2] != 0.0 || !std::isfinite(est)) return BAH_ERR_NONFINITE;
            if (est <= rtol || c.histat[1] <= 1e-14 * bn) break;
        }
        // e += Z y, then the true residual s - M e
        int* hj = reinterpret_cast<int*>(c.histat + 4);
        *hj = jd;
        BAH_CUDA_TRY(cudaMemcpyAsync(c.ijk, hj, sizeof(int), cudaMemcpyHostToDevice, st));
        launch_triangular_solve(c.iH, m + 1, c.igv, c.ijk, c.iy, 1, ks, st);
        launch_update_x<double2>(c.iZ, c.ijk, c.iy, e, np, 1, ks, st);
        launch_block_apply64(c.f5x, b, e, c.iR, s, st);
        launch_norm2(c.iR, np, c.idpart, c.inrm, 0, 1, ks, st);
        BAH_CUDA_TRY(cudaGetLastError());
        TRY(read_dev_double(c, c.inrm, &beta, st));
        if (!std::isfinite(beta)) return BAH_ERR_NONFINITE;
    }
    c.block_iters += total;
    return BAH_OK;
}

// z = P^{-1} D r with every block solved (r: one padded vector, FP64 or
// double-float; z: FP64): t_p = B r_u - A_p r_p, H_p e_p = t_p,
// s_u = r_u - B^T e_p, A_k e_k = s_k (Eq. 3.1-3.5)
template <class RIN>
static int precond_exact(Ctx& c, const RIN* r, double2* z, cudaStream_t st) {
    NvtxRange nv("exact-block preconditioner");
    const size_t np = c.np;
    const double ihx = 1.0 / c.h1, ihz = 1.0 / c.h2;
    auto solve = [&](int b, const double2* s, double2* e) {
        return c.mode == BAH_MIXED ? block_solve<BAH_MIXED>(c, b, s, e, st) : block_solve<BAH_FP64>(c, b, s, e, st);
    };
    launch_distributor<BAH_FP64, RIN>(c.n1, c.n2, ihx, ihz, c.f5x, r, c.etp, st, 1, RhsStride());
    TRY(solve(2, c.etp, z + 2 * np));
    launch_u_rhs<BAH_FP64, RIN>(c.n1, c.n2, ihx, ihz, r, z + 2 * np, c.esu, c.esu + np, st, 1, RhsStride());
    TRY(solve(0, c.esu, z));
    TRY(solve(1, c.esu + np, z + np));
    return BAH_OK;
}

template <class RIN>
static void precond_any(Ctx& c, const RIN* r, size_t rstride, void* z, size_t zstride, const Batch& bt,
                        cudaStream_t st) {
    if (c.exact) {
        // one right-hand side (rhs_block = 1 with exact blocks); the FP64 result is
        // rounded once to the flexible basis' precision in mixed mode
        if (c.exact_status != BAH_OK) return;
        double2* zz = c.mode == BAH_MIXED ? c.ez : (double2*)z;
        const int s = precond_exact<RIN>(c, r, zz, st);
        if (s != BAH_OK) { c.exact_status = s; return; }
        if (c.mode == BAH_MIXED) launch_convert<double2, float2>(c.ez, (float2*)z, c.vec_len(), st);
        return;
    }
    if constexpr (std::is_same<RIN, double2>::value) {
        if (c.dim == 3) {
            for (int k = 0; k < bt.nr; ++k) {
                if (c.mode == BAH_MIXED)
                    MG3<BAH_MIXED>::precond(c, r + k * rstride, (float2*)z + k * zstride, st);
                else
                    MG3<BAH_FP64>::precond(c, r + k * rstride, (double2*)z + k * zstride, st);
            }
            return;
        }
    }
    if (c.mode == BAH_MIXED) MG<BAH_MIXED>::template precond<RIN>(c, r, rstride, (float2*)z, zstride, bt, st);
    else MG<BAH_FP64>::template precond<RIN>(c, r, rstride, (double2*)z, zstride, bt, st);
}
// algorithmic bytes of one operator apply: input (3 components), FP64
// output, coefficients cx, nx (z-aliases when h1 == h2), d1, d2, 1/(lambda+mu)
static double op_bytes(const Ctx& c, double in_bytes, bool residual) {
    const double coef = (c.h1 == c.h2 ? 16.0 : 32.0) + 32.0 + 8.0;
    return (double)c.np * (3.0 * in_bytes + 48.0 + coef + (residual ? 48.0 : 0.0));
}
// 3-D: input (4 components), FP64 output, mu, three edge means, three complex
// diagonals, 1/(lambda+mu)
static double op_bytes3(const Ctx& c, double in_bytes, bool residual) {
    return (double)c.np * (4.0 * in_bytes + 64.0 + 88.0 + (residual ? 64.0 : 0.0));
}
// y = H x (b null) or y = b - H x on nr right-hand sides at the given element strides
static void apply_h(Ctx& c, const double2* x, size_t sx, double2* y, size_t sy, const double2* b, size_t sb, int conj,
                    int nr, cudaStream_t st, const int* active = nullptr) {
    if (c.dim == 3) {
        launch_apply3<double2>(c.op3, x, y, b, conj, nr, sx, sy, sb, st);
        return;
    }
    RhsStride rs;
    rs.s0 = sx; rs.s1 = sy; rs.s2 = sb; rs.active = active;
    launch_elastic_apply<double2>(c.op, x, y, b, conj, st, nr, rs);
}
static void op_apply_z(Ctx& c, const void* z, size_t zstride, void* y, size_t ystride, const Batch& bt,
                       cudaStream_t st) {
    if (c.dim == 3) {
        Prof pr(c, BAH_K_OPERATOR, st, bt.nr * op_bytes3(c, (double)c.vsz, false));
        if (c.mode == BAH_MIXED)
            launch_apply3<float2>(c.op3, (const float2*)z, (double2*)y, nullptr, 0, bt.nr, zstride, ystride, 0, st);
        else
            launch_apply3<double2>(c.op3, (const double2*)z, (double2*)y, nullptr, 0, bt.nr, zstride, ystride, 0, st);
        return;
    }
    Prof pr(c, BAH_K_OPERATOR, st, bt.nr * op_bytes(c, (double)c.vsz, false));
    RhsStride rs;
    rs.s0 = zstride; rs.s1 = ystride; rs.active = bt.active;
    if (c.kdf) {
        if (c.mode == BAH_MIXED && c.opdf_ok) launch_elastic_apply_dfa(c.opdf, (const float2*)z, (float4*)y, st, bt.nr, rs);
        else if (c.mode == BAH_MIXED) launch_elastic_apply_df<float2>(c.op, (const float2*)z, (float4*)y, st, bt.nr, rs);
        else launch_elastic_apply_df<double2>(c.op, (const double2*)z, (float4*)y, st, bt.nr, rs);
    } else {
        if (c.mode == BAH_MIXED && c.opdf_ok) launch_elastic_apply_dfa(c.opdf, (const float2*)z, (double2*)y, st, bt.nr, rs);
        else if (c.mode == BAH_MIXED) launch_elastic_apply<float2>(c.op, (const float2*)z, (double2*)y, nullptr, 0, st, bt.nr, rs);
        else launch_elastic_apply<double2>(c.op, (const double2*)z, (double2*)y, nullptr, 0, st, bt.nr, rs);
    }
}

// FGMRES workspace for nbatch right-hand sides: bases V (FP64 or
// double-float) and Z (the preconditioner's precision), Hessenberg matrices,
// rotations, reduction partials, status slots and the per-step graphs
static int alloc_krylov(Ctx& c, cudaStream_t st) {
    const size_t n = c.vec_len();
    const int m = c.m;
    const size_t nbt = c.nbatch;
    const size_t so = m + 2;
    TRY(c.alloc_t(&c.V, n * (m + 1) * nbt));
    TRY(c.alloc(&c.Z, n * m * c.vsz * nbt));
    TRY(c.alloc_t(&c.W, n * nbt)); TRY(c.alloc_t(&c.R, n * nbt)); TRY(c.alloc_t(&c.Bs, n * nbt));
    TRY(c.alloc_t(&c.X, n * nbt));
    TRY(c.alloc(&c.ztmp, n * c.vsz));
    TRY(c.alloc_t(&c.Hm, (size_t)(m + 1) * m * nbt));
    TRY(c.alloc_t(&c.h1v, so * nbt)); TRY(c.alloc_t(&c.h2v, so * nbt));
    TRY(c.alloc_t(&c.gsflag, nbt));
    TRY(c.alloc_t(&c.cs, so * nbt)); TRY(c.alloc_t(&c.sn, so * nbt)); TRY(c.alloc_t(&c.g, so * nbt));
    TRY(c.alloc_t(&c.y, so * nbt));
    TRY(c.alloc_t(&c.partial, so * RED_CTAS * nbt));
    TRY(c.alloc_t(&c.dpart, (size_t)RED_CTAS * nbt));
    TRY(c.alloc_t(&c.nrm, 8 * nbt));
    TRY(c.alloc_t(&c.status, 4 * nbt));
    TRY(c.alloc_t(&c.active, nbt));
    TRY(c.alloc_t(&c.jk, nbt));
    BAH_CUDA_TRY(cudaMemsetAsync(c.nrm, 0, 8 * nbt * sizeof(double), st));
    BAH_CUDA_TRY(cudaMallocHost((void**)&c.hstatus, (4 * (size_t)(m + 1) * nbt + 8 * nbt) * sizeof(double)));
    BAH_CUDA_TRY(cudaMallocHost((void**)&c.hint, kIntSlots * nbt * sizeof(int)));
    c.ks.sv = (size_t)(m + 1) * n; c.ks.sw = n; c.ks.sp = so * RED_CTAS; c.ks.so = so;
    c.ks.sh = (size_t)(m + 1) * m; c.ks.sz = (size_t)m * n; c.ks.sx = n; c.ks.active = c.active;
    BAH_CUDA_TRY(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    c.ig.assign(m, Ctx::IterGraph());
    c.itev.assign(m, nullptr);
    for (int j = 0; j < m; ++j) BAH_CUDA_TRY(cudaEventCreateWithFlags(&c.itev[j], cudaEventDisableTiming));
    if (const char* e = getenv("BAH_NO_GRAPHS")) c.use_graphs = (e[0] == '0');
    return BAH_OK;
}

// ---------------------------------------------------------------------------
// context construction
// ---------------------------------------------------------------------------
static int build(Ctx& c, const bah_medium* med, cudaStream_t st) {
    NvtxRange nv("bah setup (2-D)");
    const int np = c.np;
    const size_t cs = c.mode == BAH_MIXED ? 2 : 8, ccs = c.mode == BAH_MIXED ? 4 : 16;
    // medium upload
    double *lam, *mu, *rho, *gam;
    TRY(c.alloc_t(&lam, np)); TRY(c.alloc_t(&mu, np)); TRY(c.alloc_t(&rho, np)); TRY(c.alloc_t(&gam, np));
    BAH_CUDA_TRY(cudaMemcpyAsync(lam, med->lambda, np * sizeof(double), cudaMemcpyHostToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(mu, med->mu, np * sizeof(double), cudaMemcpyHostToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(rho, med->rho, np * sizeof(double), cudaMemcpyHostToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(gam, med->gamma, np * sizeof(double), cudaMemcpyHostToDevice, st));
    TRY(c.alloc_t(&c.cx, np)); TRY(c.alloc_t(&c.cz, np)); TRY(c.alloc_t(&c.nx, np)); TRY(c.alloc_t(&c.nz, np));
    TRY(c.alloc_t(&c.wx, np)); TRY(c.alloc_t(&c.wz, np)); TRY(c.alloc_t(&c.cinv, np));
    TRY(c.alloc_t(&c.d1, np)); TRY(c.alloc_t(&c.d2, np)); TRY(c.alloc_t(&c.dAp, np));
    for (int b = 0; b < 3; ++b) TRY(c.alloc_t(&c.dg[b], np));
    c.gam = gam;
    launch_medium_prep(c.n1, c.n2, c.h1, c.h2, c.omega, c.alpha, lam, mu, rho, gam, c.cx, c.cz, c.nx, c.nz, c.wx,
                       c.wz, c.d1, c.d2, c.cinv, c.dg[0], c.dg[1], c.dg[2], c.dAp, st);
    BAH_CUDA_TRY(cudaGetLastError());
    c.op = OpCoef{c.n1, c.n2, c.cx, c.cz, c.nx, c.nz, c.d1, c.d2, c.cinv, 1.0 / c.h1, 1.0 / c.h2};
    // double-float copies of the operator coefficients for w = H z on the FP32
    // flexible basis in mixed mode (BAH_OP_F64=1 keeps the FP64 kernel)
    {
        bool on = c.mode == BAH_MIXED;
        if (const char* e = getenv("BAH_OP_F64")) on = on && e[0] != '1';
        if (on) {
            const size_t np = c.np;
            auto conv = [&](const double* src, const float2** dst, const double* alias_of, const float2* alias_dst) {
                if (src == alias_of && alias_dst) { *dst = alias_dst; return BAH_OK; }
                float2* d = nullptr;
                TRY(c.alloc_t(&d, np));
                launch_to_df(src, d, np, st);
                *dst = d;
                return BAH_OK;
            };
            OpCoefDF& o = c.opdf;
            o.n1 = c.n1; o.n2 = c.n2;
            TRY(conv(c.cx, &o.cx, nullptr, nullptr));
            TRY(conv(c.nx, &o.nx, nullptr, nullptr));
            TRY(conv(c.cz, &o.cz, c.cx, o.cx));
            TRY(conv(c.nz, &o.nz, c.nx, o.nx));
            TRY(conv(c.cinv, &o.cinv, nullptr, nullptr));
            float4* d1 = nullptr;
            float4* d2 = nullptr;
            TRY(c.alloc_t(&d1, np));
            TRY(c.alloc_t(&d2, np));
            launch_to_df_c(c.d1, d1, np, st);
            launch_to_df_c(c.d2, d2, np, st);
            o.d1 = d1; o.d2 = d2;
            auto dfh = [](double v) {
                const float hi = (float)v;
                return make_float2(hi, (float)(v - (double)hi));
            };
            o.ihx = dfh(1.0 / c.h1);
            o.ihz = dfh(1.0 / c.h2);
            BAH_CUDA_TRY(cudaGetLastError());
            c.opdf_ok = true;
        }
    }

    // level-0 coefficients in storage precision
    const bool iso = c.h1 == c.h2;
    TRY(c.alloc(&c.s_cx, np * cs)); TRY(c.alloc(&c.s_nx, np * cs)); TRY(c.alloc(&c.s_wx, np * cs));
    launch_round_real(c.cx, c.s_cx, np, c.mode, st);
    launch_round_real(c.nx, c.s_nx, np, c.mode, st);
    launch_round_real(c.wx, c.s_wx, np, c.mode, st);
    if (iso) {
        c.s_cz = c.s_cx; c.s_nz = c.s_nx; c.s_wz = c.s_wx;
    } else {
        TRY(c.alloc(&c.s_cz, np * cs)); TRY(c.alloc(&c.s_nz, np * cs)); TRY(c.alloc(&c.s_wz, np * cs));
        launch_round_real(c.cz, c.s_cz, np, c.mode, st);
        launch_round_real(c.nz, c.s_nz, np, c.mode, st);
        launch_round_real(c.wz, c.s_wz, np, c.mode, st);
    }
    for (int b = 0; b < 3; ++b) {
        TRY(c.alloc(&c.s_dg[b], np * ccs));
        launch_round_cplx(c.dg[b], c.s_dg[b], np, c.mode, st);
    }
    TRY(c.alloc(&c.s_dAp, np * ccs));
    launch_round_cplx(c.dAp, c.s_dAp, np, c.mode, st);

    // hierarchy: level grids, FP64 stencils, Galerkin products, storage copies
    c.ln1.assign(c.L, 0); c.ln2.assign(c.L, 0);
    c.s64.assign(c.L, {}); c.sst.assign(c.L, {nullptr, nullptr, nullptr});
    for (int l = 0; l < c.L; ++l) { c.ln1[l] = c.n1 >> l; c.ln2[l] = c.n2 >> l; }
    for (int b = 0; b < 3; ++b) {
        StencilF64& s0 = c.s64[0][b];
        s0.rx = 1; s0.rz = 1; s0.n1 = c.n1; s0.n2 = c.n2;
        TRY(c.alloc_t(&s0.S, (size_t)9 * np));
        launch_fine_stencil(b, c.n1, c.n2, c.cx, c.cz, c.nx, c.nz, c.wx, c.wz, c.dg[b], s0.S, st);
        for (int l = 1; l < c.L; ++l) {
            StencilF64& s = c.s64[l][b];
            const bool bil = c.o.intergrid == BAH_INTERGRID_BILINEAR;
            s.rx = (b == 0) ? 1 : (bil ? 2 : 1);
            s.rz = (b == 1) ? 1 : (bil ? 2 : 1);
            s.n1 = c.ln1[l]; s.n2 = c.ln2[l];
            const size_t ns = (size_t)(2 * s.rx + 1) * (2 * s.rz + 1) * s.n1 * s.n2;
            TRY(c.alloc_t(&s.S, ns));
            launch_galerkin(b, c.o.intergrid, c.s64[l - 1][b], s, st);
            if (l < c.L - 1) {
                TRY(c.alloc(&c.sst[l][b], ns * ccs));
                launch_round_cplx(s.S, c.sst[l][b], ns, c.mode, st);
            }
        }
    }
    BAH_CUDA_TRY(cudaGetLastError());
    // coarsest-level inverses
    {
        NvtxRange nvi("coarsest inverses");
        const int nc = c.ln1[c.L - 1] * c.ln2[c.L - 1];
        void* work;
        int* flag;
        TRY(c.alloc(&work, ((size_t)nc * nc + nc) * sizeof(double2)));
        TRY(c.alloc_t(&flag, 1));
        for (int b = 0; b < 3; ++b) {
            TRY(c.alloc_t(&c.inv[b], (size_t)nc * nc));
            TRY(coarse_invert(b, c.s64[c.L - 1][b], c.inv[b], (double2*)work, flag, st));
        }
    }
    // multigrid vectors
    c.vX.assign(c.L, {nullptr, nullptr, nullptr});
    c.vB = c.vX; c.vT = c.vX;
    for (int l = 0; l < c.L; ++l)
        for (int b = 0; b < 3; ++b) {
            const size_t bytes = (size_t)c.ln1[l] * c.ln2[l] * c.vsz * c.nbatch;
            TRY(c.alloc(&c.vX[l][b], bytes));
            TRY(c.alloc(&c.vB[l][b], bytes));
            TRY(c.alloc(&c.vT[l][b], bytes));
            BAH_CUDA_TRY(cudaMemsetAsync(c.vX[l][b], 0, bytes, st));
            BAH_CUDA_TRY(cudaMemsetAsync(c.vB[l][b], 0, bytes, st));
            BAH_CUDA_TRY(cudaMemsetAsync(c.vT[l][b], 0, bytes, st));
        }
    {
        int dev = 0;
        BAH_CUDA_TRY(cudaGetDevice(&dev));
        BAH_CUDA_TRY(cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    // shared-memory cluster multigrid (mixed mode; BAH_SMEM_MG=0 turns it off):
    // from the first level below the fine grid whose levels, down to the
    // coarsest, fit in the shared memory of one cluster (16 CTAs, else 8)
    if (c.mode == BAH_MIXED && c.L >= 3 && c.L <= kMaxLevels) {
        bool on = true;
        if (const char* e = getenv("BAH_SMEM_MG")) on = e[0] != '0';
        int dev = 0, optin = 0;
        BAH_CUDA_TRY(cudaGetDevice(&dev));
        BAH_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        for (int l0 = 1; on && l0 < c.L - 1 && c.sm_l0 == 0; ++l0) {
            const int nlev = c.L - l0;
            int n1s[kMaxLevels], n2s[kMaxLevels], ns[kMaxLevels], rm = 1;
            for (int k = 0; k < nlev; ++k) {
                n1s[k] = c.ln1[l0 + k]; n2s[k] = c.ln2[l0 + k];
                ns[k] = 0;
                for (int b = 0; b < 3; ++b) {
                    ns[k] = std::max(ns[k], (2 * c.s64[l0 + k][b].rx + 1) * (2 * c.s64[l0 + k][b].rz + 1));
                    rm = std::max(rm, std::max(c.s64[l0 + k][b].rx, c.s64[l0 + k][b].rz));
                }
            }
            if (rm > 2) continue;                      // the kernel's stencil radius is at most 2
            for (int cs = 16; cs >= 8 && c.sm_l0 == 0; cs /= 2) {
                SmArgs a;
                std::memset(&a, 0, sizeof(a));
                const size_t bytes = smmg_layout(a, n1s, n2s, ns, nlev, cs);
                if (bytes > (size_t)optin) continue;
                if (smmg_prepare(rm, cs, bytes) >= 1) {
                    c.sm_l0 = l0; c.sm_cs = cs; c.sm_rm = rm; c.sm_bytes = bytes;
                }
            }
        }
    }
    TRY(alloc_krylov(c, st));
    if (c.o.block_krylov) {
        const size_t sq = (size_t)(c.m + 1) * c.nbatch * c.nbatch;
        TRY(c.alloc_t(&c.bC, sq)); TRY(c.alloc_t(&c.bT, (size_t)c.nbatch * c.nbatch));
        TRY(c.alloc_t(&c.bpart, sq * RED_CTAS));
        BAH_CUDA_TRY(cudaMallocHost((void**)&c.bhost, sq * sizeof(double2)));
        block_kernels_smem((size_t)(c.m + 1) * c.nbatch * c.nbatch * sizeof(double2));
    }
    if (c.exact) {
        // the blocks solved exactly: the fine operators of Eq. 2.6 / 3.4 with their
        // diagonals shifted by block_alpha (a second medium preparation, of which
        // only the three block diagonals are kept), FP64 coefficients throughout
        double2* dgb[3];
        for (int b = 0; b < 3; ++b) TRY(c.alloc_t(&dgb[b], np));
        {
            void* scratch = nullptr;
            BAH_CUDA_TRY(cudaMalloc(&scratch, (size_t)np * (7 * sizeof(double) + 3 * sizeof(double2))));
            double* sd = (double*)scratch;
            double2* sc2 = (double2*)(sd + 7 * (size_t)np);
            launch_medium_prep(c.n1, c.n2, c.h1, c.h2, c.omega, c.o.block_alpha, lam, mu, rho, gam, sd, sd + np,
                               sd + 2 * (size_t)np, sd + 3 * (size_t)np, sd + 4 * (size_t)np, sd + 5 * (size_t)np,
                               sc2, sc2 + np, sd + 6 * (size_t)np, dgb[0], dgb[1], dgb[2], sc2 + 2 * (size_t)np, st);
            cudaError_t e1 = cudaStreamSynchronize(st);
            cudaFree(scratch);
            BAH_CUDA_TRY(e1);
        }
        c.f5x = Fine5<double, double2>{c.n1, c.n2, c.cx, c.cz, c.nx, c.nz, c.wx, c.wz, dgb[0], dgb[1], dgb[2], c.dAp};
        const size_t so = c.mi + 2;
        TRY(c.alloc_t(&c.iV, (size_t)(c.mi + 1) * np)); TRY(c.alloc_t(&c.iZ, (size_t)c.mi * np));
        TRY(c.alloc_t(&c.iW, np)); TRY(c.alloc_t(&c.iR, np));
        TRY(c.alloc_t(&c.iH, (size_t)(c.mi + 1) * c.mi));
        TRY(c.alloc_t(&c.ih1, so)); TRY(c.alloc_t(&c.ih2, so)); TRY(c.alloc_t(&c.ics, so)); TRY(c.alloc_t(&c.isn, so));
        TRY(c.alloc_t(&c.igv, so)); TRY(c.alloc_t(&c.iy, so));
        TRY(c.alloc_t(&c.ipart, so * RED_CTAS)); TRY(c.alloc_t(&c.idpart, (size_t)RED_CTAS));
        TRY(c.alloc_t(&c.inrm, 8)); TRY(c.alloc_t(&c.istatus, 4)); TRY(c.alloc_t(&c.iflag, 1)); TRY(c.alloc_t(&c.ijk, 1));
        TRY(c.alloc_t(&c.ez, 3 * (size_t)np)); TRY(c.alloc_t(&c.etp, np)); TRY(c.alloc_t(&c.esu, 2 * (size_t)np));
        BAH_CUDA_TRY(cudaMemsetAsync(c.inrm, 0, 8 * sizeof(double), st));
        BAH_CUDA_TRY(cudaMallocHost((void**)&c.histat, 16 * sizeof(double)));
        c.use_graphs = false;             // the block solves read their status on the host
    }
    if (const char* e = getenv("BAH_STAGED")) c.staged = (e[0] != '0');
    if (const char* e = getenv("BAH_DGKS_ETA2")) c.dgks_eta2 = atof(e);
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    // the raw medium is no longer needed
    return BAH_OK;
}

// ---------------------------------------------------------------------------
// three-dimensional context: medium, fine stencils, Galerkin hierarchy with
// the mixed intergrid, coarsest inverses, multigrid vectors, Krylov workspace
// ---------------------------------------------------------------------------
static int build3(Ctx& c, const bah_medium* med, cudaStream_t st) {
    NvtxRange nv("bah setup (3-D)");
    const size_t np = c.np;
    double *lam, *mu, *rho, *gam, *cinv, *mue[3];
    double2 *mrt, *dg[3];
    TRY(c.alloc_t(&lam, np)); TRY(c.alloc_t(&mu, np)); TRY(c.alloc_t(&rho, np)); TRY(c.alloc_t(&gam, np));
    BAH_CUDA_TRY(cudaMemcpyAsync(lam, med->lambda, np * sizeof(double), cudaMemcpyHostToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(mu, med->mu, np * sizeof(double), cudaMemcpyHostToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(rho, med->rho, np * sizeof(double), cudaMemcpyHostToDevice, st));
    BAH_CUDA_TRY(cudaMemcpyAsync(gam, med->gamma, np * sizeof(double), cudaMemcpyHostToDevice, st));
    TRY(c.alloc_t(&cinv, np)); TRY(c.alloc_t(&mrt, np));
    for (int e = 0; e < 3; ++e) { TRY(c.alloc_t(&mue[e], np)); TRY(c.alloc_t(&dg[e], np)); }
    c.gam = gam;
    Op3& o = c.op3;
    o.n[0] = c.n1; o.n[1] = c.n2; o.n[2] = c.n3;
    const double h[3] = {c.h1, c.h2, c.h3};
    for (int a = 0; a < 3; ++a) { o.ih[a] = 1.0 / h[a]; o.ih2[a] = 1.0 / (h[a] * h[a]); }
    o.muc = mu; o.cinv = cinv; o.mrt = mrt;
    for (int e = 0; e < 3; ++e) { o.mue[e] = mue[e]; o.dg[e] = dg[e]; }
    // level grids and FP64 stencils
    c.d3.assign(c.L, {0, 0, 0});
    for (int l = 0; l < c.L; ++l) c.d3[l] = {c.n1 >> l, c.n2 >> l, c.n3 >> l};
    auto pts = [&](int l) { return (size_t)c.d3[l][0] * c.d3[l][1] * c.d3[l][2]; };
    c.s3.assign(c.L, {nullptr, nullptr, nullptr, nullptr});
    c.s3s.assign(c.L, {nullptr, nullptr, nullptr, nullptr});
    for (int q = 0; q < 4; ++q) TRY(c.alloc_t(&c.s3[0][q], 7 * np));
    launch_prep3(o, c.omega, c.alpha, lam, mu, rho, gam, cinv, mrt, mue, dg, c.s3[0].data(), st);
    int* err;
    TRY(c.alloc_t(&err, 2));
    BAH_CUDA_TRY(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
    for (int l = 1; l < c.L; ++l)
        for (int q = 0; q < 4; ++q) {
            TRY(c.alloc_t(&c.s3[l][q], 27 * pts(l)));
            launch_galerkin3(q, c.d3[l - 1].data(), l == 1 ? 7 : 27, c.s3[l - 1][q], c.s3[l][q], err, st);
        }
    for (int l = 0; l + 1 < c.L; ++l)
        for (int q = 0; q < 4; ++q) {
            const size_t cnt = (l == 0 ? 7 : 27) * pts(l);
            if (c.mode == BAH_MIXED) {
                // the mixed cycle's stencils in bfloat16 (entries rounded once from FP64)
                TRY(c.alloc(&c.s3s[l][q], cnt * sizeof(__nv_bfloat162)));
                launch_round_cplx(c.s3[l][q], c.s3s[l][q], cnt, BAH_MIXED, st);
            } else {
                c.s3s[l][q] = c.s3[l][q];
            }
        }
    BAH_CUDA_TRY(cudaGetLastError());
    int herr = 0;
    BAH_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        set_error("3-D Galerkin product produced a coupling beyond one coarse point");
        return BAH_ERR_CUDA;
    }
    // coarsest inverses
    {
        const size_t nc = pts(c.L - 1);
        void* work;
        TRY(c.alloc(&work, (nc * nc + nc) * sizeof(double2)));
        for (int q = 0; q < 4; ++q) {
            TRY(c.alloc_t(&c.inv3[q], nc * nc));
            TRY(coarse_invert3(q, c.d3[c.L - 1].data(), c.s3[c.L - 1][q], c.inv3[q], (double2*)work, err + 1, st));
        }
    }
    // multigrid vectors
    c.v3X.assign(c.L, {nullptr, nullptr, nullptr, nullptr});
    c.v3B = c.v3X; c.v3T = c.v3X;
    for (int l = 0; l < c.L; ++l)
        for (int q = 0; q < 4; ++q) {
            const size_t bytes = pts(l) * c.vsz;
            TRY(c.alloc(&c.v3X[l][q], bytes)); TRY(c.alloc(&c.v3B[l][q], bytes)); TRY(c.alloc(&c.v3T[l][q], bytes));
            BAH_CUDA_TRY(cudaMemsetAsync(c.v3X[l][q], 0, bytes, st));
            BAH_CUDA_TRY(cudaMemsetAsync(c.v3B[l][q], 0, bytes, st));
            BAH_CUDA_TRY(cudaMemsetAsync(c.v3T[l][q], 0, bytes, st));
        }
    TRY(alloc_krylov(c, st));
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    return BAH_OK;
}

// ---------------------------------------------------------------------------
// FGMRES, nbatch right-hand sides in lockstep (device vectors b, x with
// stride n; b sanitised).  Every right-hand side has its own Krylov basis,
// Hessenberg matrix and rotations; the kernels of one step serve all of them
// and skip the inactive ones.
// ---------------------------------------------------------------------------
static double* status_slot(Ctx& c, int j) { return c.hstatus + 4 * (size_t)j * c.nbatch; }
static double* scalar_slot(Ctx& c) { return c.hstatus + 4 * (size_t)(c.m + 1) * c.nbatch; }

// copy sc[r*8 + slot] of every right-hand side to the host (synchronises)
static int read_scalars(Ctx& c, int slot, double* out, cudaStream_t st) {
    double* h = scalar_slot(c);
    BAH_CUDA_TRY(cudaMemcpy2DAsync(h, sizeof(double), c.nrm + slot, 8 * sizeof(double), sizeof(double), c.nbatch,
                                   cudaMemcpyDeviceToHost, st));
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    for (int r = 0; r < c.nbatch; ++r) out[r] = h[r];
    return BAH_OK;
}
// Host-to-device copy of one int per right-hand side through a ring of
// pinned staging slots: at most a few uploads happen between two waits on
// the stream, so a slot's copy has completed before the slot comes round again.
static int upload_ints(Ctx& c, const std::vector<int>& v, int* dev, int /*which*/, cudaStream_t st) {
    int* h = c.hint + (size_t)(c.hint_slot++ % kIntSlots) * c.nbatch;
    for (int r = 0; r < c.nbatch; ++r) h[r] = v[r];
    BAH_CUDA_TRY(cudaMemcpyAsync(dev, h, c.nbatch * sizeof(int), cudaMemcpyHostToDevice, st));
    return BAH_OK;
}

// One FGMRES step j for all right-hand sides (everything between two status
// reads): z_j = P^{-1} D v_j, w = H z_j, Gram-Schmidt with selective
// reorthogonalisation, Givens update, v_{j+1} = w / ||w||, and the copy of
// the step's status to pinned slot j.
static void iter_body(Ctx& c, int j, cudaStream_t st) {
    const size_t n = c.vec_len();
    const int m = c.m, nb = c.nbatch;
    const KS& ks = c.ks;
    Batch bt;
    bt.nr = nb;
    bt.active = c.active;
    void* zj = (char*)c.Z + (size_t)j * n * c.vsz;
    float4* Vd = (float4*)c.V;
    float4* Wd = (float4*)c.W;
    if (c.kdf) precond_any(c, Vd + (size_t)j * n, ks.sv, zj, ks.sz, bt, st);
    else precond_any(c, c.V + (size_t)j * n, ks.sv, zj, ks.sz, bt, st);
    op_apply_z(c, zj, ks.sz, c.W, n, bt, st);
    const double k1 = j + 1;
    {
        Prof pr(c, BAH_K_DOT, st, nb * (k1 + 1) * n * 16.0, 2);
        if (c.kdf) launch_dot_norm_df(Vd, j + 1, Wd, n, c.partial, c.h1v, nullptr, nb, ks, st);
        else launch_dot_norm(c.V, j + 1, c.W, n, c.partial, c.h1v, nullptr, nb, ks, st);
    }
    {
        Prof pr(c, BAH_K_AXPY, st, nb * (k1 + 2) * n * 16.0);
        if (c.kdf) launch_axpy_norm_df(Vd, j + 1, c.h1v, Wd, n, c.dpart, nullptr, nb, ks, st);
        else launch_axpy_norm(c.V, j + 1, c.h1v, c.W, n, c.dpart, nullptr, nb, ks, st);
    }
    {
        Prof pr(c, BAH_K_NORM, st, 0.0);
        launch_dgks_decide(c.dpart, c.h1v, j + 1, c.gsflag, c.nrm, nb, ks, st, c.dgks_eta2);
    }
    {
        Prof pr(c, BAH_K_DOT, st, 0.0, 2);      // runs only where the flag is set (bytes counted as zero)
        if (c.kdf) launch_dot_norm_df(Vd, j + 1, Wd, n, c.partial, c.h2v, c.gsflag, nb, ks, st);
        else launch_dot_norm(c.V, j + 1, c.W, n, c.partial, c.h2v, c.gsflag, nb, ks, st);
    }
    {
        Prof pr(c, BAH_K_AXPY, st, 0.0);
        if (c.kdf) launch_axpy_norm_df(Vd, j + 1, c.h2v, Wd, n, c.dpart, c.gsflag, nb, ks, st);
        else launch_axpy_norm(c.V, j + 1, c.h2v, c.W, n, c.dpart, c.gsflag, nb, ks, st);
    }
    {
        Prof pr(c, BAH_K_SMALL, st, nb * n * 32.0, 3);
        launch_pass2_norm(c.dpart, c.gsflag, c.nrm, nb, ks, st);
        launch_arnoldi_givens(c.Hm, m + 1, c.h1v, c.h2v, c.nrm, j, c.cs, c.sn, c.g, c.status, nb, ks, st);
        if (c.kdf) launch_scale_copy_df(c.W, false, c.nrm, 2, Vd + (size_t)(j + 1) * n, n, n, ks.sv, nb, ks, st);
        else launch_scale_copy(c.W, c.nrm, 2, c.V + (size_t)(j + 1) * n, n, n, ks.sv, nb, ks, st);
    }
    cudaMemcpyAsync(status_slot(c, j), c.status, 4 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, st);
}

static int ensure_graph(Ctx& c, int j) {
    Ctx::IterGraph& G = c.ig[j];
    if (G.exec && G.mask == c.tmask) return BAH_OK;
    Ctx::clear_graph(G);
    G.mask = c.tmask;
    BAH_CUDA_TRY(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    c.capturing = &G;
    iter_body(c, j, c.cap_stream);
    c.capturing = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c.cap_stream, &g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        Ctx::clear_graph(G);
        set_error(std::string("graph capture failed: ") + cudaGetErrorString(e));
        return BAH_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        Ctx::clear_graph(G);
        set_error(std::string("graph instantiate failed: ") + cudaGetErrorString(e));
        return BAH_ERR_CUDA;
    }
    return BAH_OK;
}

static int launch_iter(Ctx& c, int j, cudaStream_t st) {
    NvtxRange nv("fgmres step");
    if (c.use_graphs) {
        int s = ensure_graph(c, j);
        if (s != BAH_OK) {
            c.use_graphs = false;     // fall back to direct launches from now on
        } else {
            Ctx::IterGraph& G = c.ig[j];
            BAH_CUDA_TRY(cudaGraphLaunch(G.exec, st));
            c.launches += G.launches;
            for (int k = 0; k < 16; ++k) {
                c.cls_launch[k] += G.cls_launch[k];
                c.cls_calls[k] += G.cls_calls[k];
                c.cls_bytes[k] += G.cls_bytes[k];
            }
        }
    }
    if (!c.use_graphs) iter_body(c, j, st);
    BAH_CUDA_TRY(cudaEventRecord(c.itev[j], st));
    return BAH_OK;
}

static int finish_iter(Ctx& c, int j) {
    BAH_CUDA_TRY(cudaEventSynchronize(c.itev[j]));
    if (c.use_graphs && c.ig[j].exec) {
        for (auto& e : c.ig[j].ev) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e.second.first, e.second.second) == cudaSuccess) c.cls_ms[e.first] += ms;
            else cudaGetLastError();
        }
    }
    return BAH_OK;
}

static int fgmres_batch(Ctx& c, const double2* b, double2* x, int nr, double rtol, bah_stats* out, cudaStream_t st) {
    const size_t n = c.vec_len();
    const int m = c.m, nb = c.nbatch;
    const KS& ks = c.ks;
    std::vector<bah_stats> S(nb);
    std::vector<double> bn(nb, 0.0), beta(nb, 0.0), est(nb, 1.0), tmp(nb);
    std::vector<int> act(nb, 0), cyc(nb, 0), jd(nb, 0);
    for (int r = 0; r < nb; ++r) { S[r] = bah_stats{}; S[r].status = BAH_OK; act[r] = r < nr ? 1 : 0; }
    TRY(upload_ints(c, act, c.active, 0, st));
    {
        Prof pr(c, BAH_K_NORM, st, (double)nr * n * 16.0, 2);
        launch_norm2(b, n, c.dpart, c.nrm, 1, nb, ks, st);
    }
    TRY(read_scalars(c, 1, bn.data(), st));
    BAH_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)nr * n * sizeof(double2), st));
    BAH_CUDA_TRY(cudaMemcpyAsync(c.R, b, (size_t)nr * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    // beta = ||b|| (x_0 = 0)
    BAH_CUDA_TRY(cudaMemcpy2DAsync(c.nrm, 8 * sizeof(double), c.nrm + 1, 8 * sizeof(double), sizeof(double), nb,
                                   cudaMemcpyDeviceToDevice, st));
    BAH_CUDA_TRY(cudaMemset2DAsync(c.nrm + 3, 8 * sizeof(double), 0, sizeof(double), nb, st));
    for (int r = 0; r < nr; ++r) {
        beta[r] = bn[r];
        if (!std::isfinite(bn[r])) { S[r].status = BAH_ERR_NONFINITE; act[r] = 0; }
        else if (!(bn[r] > 0.0)) { act[r] = 0; }                  // b = 0: x = 0
        else if (beta[r] <= rtol * bn[r]) act[r] = 0;
    }
    int total = 0;
    auto any = [&](const std::vector<int>& v) { for (int q : v) if (q) return true; return false; };
    while (any(act) && total < c.o.maxit) {
        NvtxRange nvc("fgmres restart cycle");
        TRY(upload_ints(c, act, c.active, 0, st));
        // v_0 = r / beta, g = beta e_1
        {
            Prof pr(c, BAH_K_SMALL, st, (double)nr * n * 32.0, 2);
            if (c.kdf) launch_scale_copy_df(c.R, true, c.nrm, 0, (float4*)c.V, n, n, ks.sv, nb, ks, st);
            else launch_scale_copy(c.R, c.nrm, 0, c.V, n, n, ks.sv, nb, ks, st);
            launch_init_arnoldi(c.nrm, c.g, m, c.status, nb, ks, st);
        }
        const int mm = std::min(m, c.o.maxit - total);
        cyc = act;
        std::fill(jd.begin(), jd.end(), 0);
        TRY(launch_iter(c, 0, st));
        for (int j = 0; j < mm; ++j) {
            if (j + 1 < mm) TRY(launch_iter(c, j + 1, st));    // queued behind step j
            TRY(finish_iter(c, j));
            if (c.exact_status != BAH_OK) {
                set_error("an exact block solve failed inside the preconditioner");
                return c.exact_status;
            }
            const double* hs = status_slot(c, j);
            ++total;
            bool changed = false;
            for (int r = 0; r < nb; ++r) {
                if (!cyc[r]) continue;
                S[r].iters++;
                jd[r] = j + 1;
                est[r] = hs[4 * r] / bn[r];
                bool stop = false;
                if (hs[4 * r + 2] != 0.0 || !std::isfinite(est[r])) { S[r].status = BAH_ERR_NONFINITE; stop = true; }
                else if (est[r] <= rtol) stop = true;
                else if (hs[4 * r + 1] <= 1e-14 * bn[r]) stop = true;    // (lucky) breakdown
                if (stop) { cyc[r] = 0; changed = true; }
            }
            if (!any(cyc)) break;
            if (changed && j + 2 < mm) TRY(upload_ints(c, cyc, c.active, 0, st));   // takes effect from step j+2
        }
        // solution update and true residual for the right-hand sides of this cycle
        for (int r = 0; r < nb; ++r) if (S[r].status == BAH_ERR_NONFINITE) jd[r] = 0;
        TRY(upload_ints(c, jd, c.jk, 1, st));
        std::vector<int> upd(nb);
        for (int r = 0; r < nb; ++r) upd[r] = (act[r] && S[r].status != BAH_ERR_NONFINITE) ? 1 : 0;
        TRY(upload_ints(c, upd, c.active, 0, st));
        {
            Prof pr(c, BAH_K_SMALL, st, 0.0);
            launch_triangular_solve(c.Hm, m + 1, c.g, c.jk, c.y, nb, ks, st);
        }
        {
            double kk = 0;
            for (int r = 0; r < nb; ++r) kk += jd[r];
            Prof pr(c, BAH_K_UPDATE, st, kk * n * c.vsz + 32.0 * n * nr);
            if (c.mode == BAH_MIXED) launch_update_x<float2>((const float2*)c.Z, c.jk, c.y, x, n, nb, ks, st);
            else launch_update_x<double2>((const double2*)c.Z, c.jk, c.y, x, n, nb, ks, st);
        }
        {
            RhsStride rs;
            rs.s0 = n; rs.s1 = n; rs.s2 = n; rs.active = c.active;
            Prof pr(c, BAH_K_OPERATOR, st, nr * (c.dim == 3 ? op_bytes3(c, 16.0, true) : op_bytes(c, 16.0, true)));
            // 3-D: only the nr right-hand sides of this batch (x holds no more)
            apply_h(c, x, rs.s0, c.R, rs.s1, b, rs.s2, 0, c.dim == 3 ? nr : nb, st, rs.active);
        }
        {
            Prof pr(c, BAH_K_NORM, st, (double)nr * n * 16.0, 2);
            launch_norm2(c.R, n, c.dpart, c.nrm, 0, nb, ks, st);
        }
        BAH_CUDA_TRY(cudaGetLastError());
        TRY(read_scalars(c, 0, tmp.data(), st));
        for (int r = 0; r < nb; ++r) {
            if (!upd[r]) { act[r] = 0; continue; }
            beta[r] = tmp[r];
            S[r].restarts++;
            if (!std::isfinite(beta[r])) { S[r].status = BAH_ERR_NONFINITE; act[r] = 0; }
            else if (beta[r] <= rtol * bn[r]) act[r] = 0;
        }
        for (int r = 0; r < nb; ++r) if (S[r].status == BAH_ERR_NONFINITE) act[r] = 0;
    }
    int first = BAH_OK;
    for (int r = 0; r < nr; ++r) {
        S[r].relres_true = bn[r] > 0.0 ? beta[r] / bn[r] : 0.0;
        S[r].relres_est = bn[r] > 0.0 ? est[r] : 0.0;
        if (S[r].status == BAH_OK && !(S[r].relres_true <= rtol)) S[r].status = BAH_ERR_NOT_CONVERGED;
        if (out) out[r] = S[r];
        if (S[r].status != BAH_OK && first == BAH_OK) first = S[r].status;
    }
    return first;
}

// ---------------------------------------------------------------------------
// Block FGMRES (block_krylov = 1): one Krylov space for the batch's s
// right-hand sides.  Per step j: Z_j = M(V_j) and W = H Z_j for the s columns
// (the batched preconditioner and operator), two passes of block classical
// Gram-Schmidt C = [V_0..V_j]^H W, W -= [V_0..V_j] C on the device, the new
// block's QR by CholQR2 (the s x s Gram matrices on the device, their
// Cholesky factors on the host), and the block Hessenberg least squares
// min ||E_1 S_0 - Hbar Y||_F on the host by Householder reflections added
// block column by block column.  FP64 basis and arithmetic; the flexible
// basis Z in the multigrid's precision.  The oracle's block_fgmres follows the
// same steps.
// ---------------------------------------------------------------------------
using cdx = std::complex<double>;

// Cholesky G = L L^H of an s x s Hermitian matrix (row-major); false if not
// positive definite
static bool host_cholesky(int s, const std::vector<cdx>& G, std::vector<cdx>& L) {
    L.assign((size_t)s * s, 0.0);
    for (int j = 0; j < s; ++j) {
        double d = G[(size_t)j * s + j].real();
        for (int k = 0; k < j; ++k) d -= std::norm(L[(size_t)j * s + k]);
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * s + j] = ljj;
        for (int i = j + 1; i < s; ++i) {
            cdx v = G[(size_t)i * s + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * s + k] * std::conj(L[(size_t)j * s + k]);
            L[(size_t)i * s + j] = v / ljj;
        }
    }
    return true;
}

struct BlockWork {
    int s = 0, m = 0;
    double2* C = nullptr;        // device (m+1) s x s coefficients / Gram matrices / Y
    double2* T = nullptr;        // device s x s triangular factor
    double2* part = nullptr;     // device dot partials
    double2* hbuf = nullptr;     // pinned host staging ((m+1) s x s)
};

// One CholQR pass: G = W^H W (W: s columns at stride n), G = L L^H, and the
// columns W R^{-1} (R = L^H) written to dst (stride sd; may be W itself).
// R returned (row-major, upper triangular).
static int cholqr_pass(Ctx& c, BlockWork& bw, const double2* W, size_t n, double2* dst, size_t sd,
                       std::vector<cdx>& R, cudaStream_t st) {
    const int s = bw.s;
    launch_block_dot(W, n, 1, s, W, n, bw.part, bw.C, st);
    BAH_CUDA_TRY(cudaMemcpyAsync(bw.hbuf, bw.C, (size_t)s * s * sizeof(double2), cudaMemcpyDeviceToHost, st));
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<cdx> G((size_t)s * s), L;
    for (int q = 0; q < s * s; ++q) G[q] = cdx(bw.hbuf[q].x, bw.hbuf[q].y);     // G[a][b] = conj(w_a) . w_b
    if (!host_cholesky(s, G, L)) {
        set_error("block FGMRES: the new block is numerically rank deficient (Cholesky QR failed)");
        return BAH_ERR_NONFINITE;
    }
    // R = L^H (upper); T = R^{-1} by back substitution, row-major T[q][b]
    R.assign((size_t)s * s, 0.0);
    for (int i = 0; i < s; ++i)
        for (int j = i; j < s; ++j) R[(size_t)i * s + j] = std::conj(L[(size_t)j * s + i]);
    std::vector<cdx> T((size_t)s * s, 0.0);
    for (int b = 0; b < s; ++b) {
        T[(size_t)b * s + b] = 1.0 / R[(size_t)b * s + b];
        for (int q = b - 1; q >= 0; --q) {
            cdx acc = 0.0;
            for (int k = q + 1; k <= b; ++k) acc += R[(size_t)q * s + k] * T[(size_t)k * s + b];
            T[(size_t)q * s + b] = -acc / R[(size_t)q * s + q];
        }
    }
    for (int q = 0; q < s * s; ++q) bw.hbuf[q] = make_double2(T[q].real(), T[q].imag());
    BAH_CUDA_TRY(cudaMemcpyAsync(bw.T, bw.hbuf, (size_t)s * s * sizeof(double2), cudaMemcpyHostToDevice, st));
    launch_block_scale(W, s, bw.T, dst, sd, n, st);
    BAH_CUDA_TRY(cudaStreamSynchronize(st));         // the staging buffer is reused next
    return BAH_OK;
}
// CholQR2: dst = Q with W = Q R (W is overwritten by the first pass)
static int cholqr2(Ctx& c, BlockWork& bw, double2* W, size_t n, double2* dst, size_t sd, std::vector<cdx>& R,
                   cudaStream_t st) {
    const int s = bw.s;
    std::vector<cdx> R1, R2;
    TRY(cholqr_pass(c, bw, W, n, W, n, R1, st));
    TRY(cholqr_pass(c, bw, W, n, dst, sd, R2, st));
    R.assign((size_t)s * s, 0.0);
    for (int i = 0; i < s; ++i)
        for (int j = i; j < s; ++j) {
            cdx acc = 0.0;
            for (int k = i; k <= j; ++k) acc += R2[(size_t)i * s + k] * R1[(size_t)k * s + j];
            R[(size_t)i * s + j] = acc;
        }
    return BAH_OK;
}

// Incremental Householder QR of the block Hessenberg matrix (column-major,
// ld rows) and of its right-hand side G = Q^H E_1 S_0
struct BlockLS {
    int s, m, ld;
    std::vector<cdx> H;      // ld x (m s)
    std::vector<cdx> G;      // ld x s
    std::vector<std::vector<cdx>> refl;   // reflector per column (from its row down)
    void init(int s_, int m_, const std::vector<cdx>& S0) {
        s = s_; m = m_; ld = (m + 1) * s;
        H.assign((size_t)ld * m * s, 0.0);
        G.assign((size_t)ld * s, 0.0);
        refl.assign((size_t)m * s, {});
        for (int i = 0; i < s; ++i)
            for (int b = 0; b < s; ++b) G[(size_t)b * ld + i] = S0[(size_t)i * s + b];
    }
    cdx& h(int i, int j) { return H[(size_t)j * ld + i]; }
    // block column j is in H (rows 0 .. (j+2)s - 1); triangularise it, return
    // the residual norm of each right-hand side column
    void add_block(int j, std::vector<double>& res) {
        const int c0 = j * s, rows = (j + 2) * s;
        for (int c = 0; c < c0; ++c) apply(c, c0, c0 + s, rows);
        for (int c = c0; c < c0 + s; ++c) {
            std::vector<cdx> v(rows - c);
            double nx = 0.0;
            for (int i = c; i < rows; ++i) { v[i - c] = h(i, c); nx += std::norm(v[i - c]); }
            nx = std::sqrt(nx);
            const cdx x0 = v[0];
            const cdx ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cdx(1.0, 0.0);
            const cdx alpha = -ph * nx;
            v[0] -= alpha;
            double nv = 0.0;
            for (const cdx& q : v) nv += std::norm(q);
            nv = std::sqrt(nv);
            if (nv > 0.0)
                for (cdx& q : v) q /= nv;
            refl[c] = v;
            apply(c, c, c0 + s, rows);
            applyG(c, rows);
        }
        res.assign(s, 0.0);
        for (int b = 0; b < s; ++b) {
            double t = 0.0;
            for (int i = (j + 1) * s; i < rows; ++i) t += std::norm(G[(size_t)b * ld + i]);
            res[b] = std::sqrt(t);
        }
    }
    void apply(int c, int col_from, int col_to, int rows) {
        const std::vector<cdx>& v = refl[c];
        if (v.empty()) return;
        const int top = std::min(rows, c + (int)v.size());
        for (int k = col_from; k < col_to; ++k) {
            cdx d = 0.0;
            for (int i = c; i < top; ++i) d += std::conj(v[i - c]) * h(i, k);
            for (int i = c; i < top; ++i) h(i, k) -= 2.0 * v[i - c] * d;
        }
    }
    void applyG(int c, int rows) {
        const std::vector<cdx>& v = refl[c];
        const int top = std::min(rows, c + (int)v.size());
        for (int b = 0; b < s; ++b) {
            cdx d = 0.0;
            for (int i = c; i < top; ++i) d += std::conj(v[i - c]) * G[(size_t)b * ld + i];
            for (int i = c; i < top; ++i) G[(size_t)b * ld + i] -= 2.0 * v[i - c] * d;
        }
    }
    // Y (k s x s, row-major [row][b]) = R^{-1} G[0 .. k s)
    void solve(int k, std::vector<cdx>& Y) {
        const int N = k * s;
        Y.assign((size_t)N * s, 0.0);
        for (int b = 0; b < s; ++b)
            for (int i = N - 1; i >= 0; --i) {
                cdx acc = G[(size_t)b * ld + i];
                for (int q = i + 1; q < N; ++q) acc -= h(i, q) * Y[(size_t)q * s + b];
                Y[(size_t)i * s + b] = acc / h(i, i);
            }
    }
};

static int fgmres_block(Ctx& c, const double2* b, double2* x, int s, double rtol, bah_stats* out, cudaStream_t st) {
    const size_t n = c.vec_len(), sv = c.ks.sv;
    const int m = c.m;
    KS ks = c.ks;
    ks.active = nullptr;
    Batch bt;
    bt.nr = s;
    bt.active = nullptr;
    BlockWork bw;
    bw.s = s; bw.m = m;
    bw.C = c.bC; bw.T = c.bT; bw.part = c.bpart; bw.hbuf = c.bhost;
    std::vector<double> bn(s), beta(s), est(s, 1.0);
    launch_norm2(b, n, c.dpart, c.nrm, 1, s, ks, st);
    {
        std::vector<double> tmp(c.nbatch);
        TRY(read_scalars(c, 1, tmp.data(), st));
        for (int r = 0; r < s; ++r) bn[r] = tmp[r];
    }
    for (int r = 0; r < s; ++r)
        if (!(bn[r] > 0.0) || !std::isfinite(bn[r])) {
            set_error("block FGMRES needs finite, nonzero right-hand sides");
            return BAH_ERR_ARG;
        }
    BAH_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)s * n * sizeof(double2), st));
    BAH_CUDA_TRY(cudaMemcpyAsync(c.R, b, (size_t)s * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    beta = bn;
    int total = 0, restarts = 0;
    std::vector<cdx> S0, R, Y;
    std::vector<double> res;
    auto done = [&]() {
        for (int r = 0; r < s; ++r) if (beta[r] > rtol * bn[r]) return false;
        return true;
    };
    while (!done() && total < c.o.maxit) {
        NvtxRange nvc("block fgmres restart cycle");
        // R_0 = V_0 S_0
        TRY(cholqr2(c, bw, c.R, n, c.V, sv, S0, st));
        BlockLS ls;
        ls.init(s, m, S0);
        const int mm = std::min(m, c.o.maxit - total);
        int jd = 0;
        for (int j = 0; j < mm; ++j) {
            void* zj = (char*)c.Z + (size_t)j * n * c.vsz;
            precond_any(c, c.V + (size_t)j * n, sv, zj, ks.sz, bt, st);
            op_apply_z(c, zj, ks.sz, c.W, n, bt, st);
            for (int pass = 0; pass < 2; ++pass) {            // block CGS2
                launch_block_dot(c.V, sv, j + 1, s, c.W, n, bw.part, bw.C, st);
                const size_t cnt = (size_t)(j + 1) * s * s;
                BAH_CUDA_TRY(cudaMemcpyAsync(bw.hbuf, bw.C, cnt * sizeof(double2), cudaMemcpyDeviceToHost, st));
                launch_block_update(c.V, sv, j + 1, s, bw.C, c.W, n, 1, st);
                BAH_CUDA_TRY(cudaStreamSynchronize(st));
                for (int row = 0; row < (j + 1) * s; ++row)
                    for (int q = 0; q < s; ++q)
                        ls.h(row, j * s + q) += cdx(bw.hbuf[(size_t)row * s + q].x, bw.hbuf[(size_t)row * s + q].y);
            }
            TRY(cholqr2(c, bw, c.W, n, c.V + (size_t)(j + 1) * n, sv, R, st));
            for (int i = 0; i < s; ++i)
                for (int q = 0; q < s; ++q) ls.h((j + 1) * s + i, j * s + q) = R[(size_t)i * s + q];
            ls.add_block(j, res);
            ++total;
            jd = j + 1;
            bool all = true;
            for (int r = 0; r < s; ++r) {
                est[r] = res[r] / bn[r];
                if (!std::isfinite(est[r])) { set_error("non-finite block residual"); return BAH_ERR_NONFINITE; }
                if (res[r] > rtol * bn[r]) all = false;
            }
            if (all) break;
        }
        // X += [Z_0 .. Z_{jd-1}] Y
        ls.solve(jd, Y);
        for (size_t q = 0; q < Y.size(); ++q) bw.hbuf[q] = make_double2(Y[q].real(), Y[q].imag());
        BAH_CUDA_TRY(cudaMemcpyAsync(bw.C, bw.hbuf, Y.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        if (c.mode == BAH_MIXED) launch_block_xupdate<float2>((const float2*)c.Z, ks.sz, jd, s, bw.C, x, n, st);
        else launch_block_xupdate<double2>((const double2*)c.Z, ks.sz, jd, s, bw.C, x, n, st);
        apply_h(c, x, n, c.R, n, b, n, 0, s, st);
        launch_norm2(c.R, n, c.dpart, c.nrm, 0, s, ks, st);
        std::vector<double> tmp(c.nbatch);
        TRY(read_scalars(c, 0, tmp.data(), st));
        for (int r = 0; r < s; ++r) {
            beta[r] = tmp[r];
            if (!std::isfinite(beta[r])) { set_error("non-finite true residual"); return BAH_ERR_NONFINITE; }
        }
        ++restarts;
    }
    int first = BAH_OK;
    for (int r = 0; r < s; ++r) {
        bah_stats q{};
        q.iters = total;
        q.restarts = restarts;
        q.relres_true = beta[r] / bn[r];
        q.relres_est = est[r];
        q.status = q.relres_true <= rtol ? BAH_OK : BAH_ERR_NOT_CONVERGED;
        if (out) out[r] = q;
        if (q.status != BAH_OK && first == BAH_OK) first = q.status;
    }
    return first;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace bah

// ===========================================================================
// C ABI
// ===========================================================================
using namespace bah;

struct bah_ctx {
    Ctx c;
};

namespace bah {
// the 2-D operator coefficients (null for a 3-D context)
const OpCoef* context_op(const bah_ctx* ctx) { return ctx->c.dim == 2 ? &ctx->c.op : nullptr; }
size_t context_vec_len(const bah_ctx* ctx) { return ctx->c.vec_len(); }
}  // namespace bah

extern "C" {

void bah_default_opts(bah_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = BAH_MIXED;
    o->levels = 0;
    o->max_coarse_cells = 256;
    o->cycle = BAH_CYCLE_V;
    o->nu_pre = 1;
    o->nu_post = 2;
    o->jacobi_w[0] = 0.8; o->jacobi_w[1] = 0.8; o->jacobi_w[2] = 0.3;
    o->n_jacobi_w = 3;
    o->shift_alpha = -1.0;
    o->intergrid = BAH_INTERGRID_BILINEAR;
    o->restart = 20;
    o->maxit = 5000;
    o->rhs_block = 1;
    o->krylov_arith = BAH_KRYLOV_FP64;
    o->block_rtol = 0.0;
    o->block_maxit = 2000;
    o->block_alpha = 0.0;
    o->block_krylov = 0;
}

const char* bah_status_string(int s) {
    switch (s) {
        case BAH_OK: return "BAH_OK";
        case BAH_ERR_ARG: return "BAH_ERR_ARG";
        case BAH_ERR_OOM: return "BAH_ERR_OOM";
        case BAH_ERR_CUDA: return "BAH_ERR_CUDA";
        case BAH_ERR_NOT_CONVERGED: return "BAH_ERR_NOT_CONVERGED";
        case BAH_ERR_NONFINITE: return "BAH_ERR_NONFINITE";
        case BAH_ERR_UNSUPPORTED: return "BAH_ERR_UNSUPPORTED";
        default: return "BAH_ERR_UNKNOWN";
    }
}

const char* bah_last_error(void) { return g_err.c_str(); }

int bah_create(const bah_grid* grid, const bah_medium* med, const bah_opts* opts, bah_ctx** out) {
    if (!out) { set_error("out is NULL"); return BAH_ERR_ARG; }
    *out = nullptr;
    g_err.clear();
    if (!grid || !med) { set_error("grid or medium is NULL"); return BAH_ERR_ARG; }
    if (grid->dim != 2 && grid->dim != 3) { set_error("dim must be 2 or 3"); return BAH_ERR_ARG; }
    const int dim = grid->dim;
    if (!med->lambda || !med->mu || !med->rho || !med->gamma) { set_error("medium array is NULL"); return BAH_ERR_ARG; }
    if (!(med->omega > 0.0)) { set_error("omega must be > 0"); return BAH_ERR_ARG; }
    for (int a = 0; a < dim; ++a)
        if (grid->n[a] < 4 || !(grid->h[a] > 0.0)) {
            set_error("need n >= 4 cells per axis and h > 0");
            return BAH_ERR_ARG;
        }
    if (dim == 3 && (long long)grid->n[0] * grid->n[1] * grid->n[2] * 4 > 2147483647LL) {
        set_error("3-D grid too large (4 * cells must fit in a 32-bit index)");
        return BAH_ERR_ARG;
    }
    bah_opts o;
    if (opts) o = *opts; else bah_default_opts(&o);
    if (o.precision != BAH_FP64 && o.precision != BAH_MIXED) { set_error("bad precision"); return BAH_ERR_ARG; }
    if (o.restart < 1 || o.restart > 64) { set_error("restart must be in 1..64"); return BAH_ERR_ARG; }
    if (o.maxit < 1) { set_error("maxit must be >= 1"); return BAH_ERR_ARG; }
    if (o.rhs_block < 1 || o.rhs_block > 256) { set_error("rhs_block must be in 1..256"); return BAH_ERR_ARG; }
    if (o.krylov_arith != BAH_KRYLOV_FP64 && o.krylov_arith != BAH_KRYLOV_DF) { set_error("bad krylov_arith"); return BAH_ERR_ARG; }
    if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre > 8 || o.nu_post > 8) { set_error("bad nu"); return BAH_ERR_ARG; }
    if (o.n_jacobi_w < 1 || o.n_jacobi_w > 8) { set_error("n_jacobi_w must be in 1..8"); return BAH_ERR_ARG; }
    if (o.intergrid != BAH_INTERGRID_BILINEAR && o.intergrid != BAH_INTERGRID_MIXED) {
        set_error("bad intergrid");
        return BAH_ERR_ARG;
    }
    if (o.cycle != BAH_CYCLE_V && o.cycle != BAH_CYCLE_W) { set_error("bad cycle"); return BAH_ERR_ARG; }
    if (!(o.block_rtol >= 0.0) || o.block_maxit < 1 || !(o.block_alpha >= 0.0)) {
        set_error("block_rtol and block_alpha must be >= 0 and block_maxit >= 1");
        return BAH_ERR_ARG;
    }
    if (o.block_krylov != 0 && o.block_krylov != 1) { set_error("bad block_krylov"); return BAH_ERR_ARG; }
    if (o.block_krylov && (dim != 2 || o.rhs_block < 2 || o.rhs_block > 16 || o.krylov_arith != BAH_KRYLOV_FP64 ||
                           o.block_rtol > 0.0)) {
        set_error("block FGMRES (block_krylov = 1) is implemented for 2-D grids, rhs_block 2..16, the FP64 basis "
                  "and multigrid block solves");
        return BAH_ERR_UNSUPPORTED;
    }
    if (o.block_rtol > 0.0 && (dim != 2 || o.rhs_block != 1)) {
        set_error("exact block solves (block_rtol > 0) are implemented for 2-D grids with rhs_block = 1");
        return BAH_ERR_UNSUPPORTED;
    }
    if (dim == 3 && o.intergrid != BAH_INTERGRID_MIXED) {
        set_error("3-D grids need intergrid = BAH_INTERGRID_MIXED (Eq. 4.4)");
        return BAH_ERR_UNSUPPORTED;
    }
    if (dim == 3 && o.krylov_arith != BAH_KRYLOV_FP64) {
        set_error("3-D grids support krylov_arith = BAH_KRYLOV_FP64 only");
        return BAH_ERR_UNSUPPORTED;
    }

    bah_ctx* h = new (std::nothrow) bah_ctx();
    if (!h) { set_error("host allocation failed"); return BAH_ERR_OOM; }
    Ctx& c = h->c;
    c.dim = dim; c.n1 = grid->n[0]; c.n2 = grid->n[1]; c.np = c.n1 * c.n2;
    c.h1 = grid->h[0]; c.h2 = grid->h[1]; c.omega = med->omega;
    if (dim == 3) { c.n3 = grid->n[2]; c.h3 = grid->h[2]; c.np *= c.n3; }
    c.o = o;
    c.mode = o.precision;
    c.vsz = c.mode == BAH_MIXED ? sizeof(float2) : sizeof(double2);
    c.m = o.restart;
    c.nbatch = o.rhs_block;
    c.kdf = o.krylov_arith == BAH_KRYLOV_DF;
    c.exact = o.block_rtol > 0.0;
    // levels
    int L = 1;
    {
        int a = c.n1, b = c.n2, d = dim == 3 ? c.n3 : 2;
        auto halvable = [&]() { return a % 2 == 0 && b % 2 == 0 && a / 2 >= 2 && b / 2 >= 2 &&
                                       (dim == 2 || (d % 2 == 0 && d / 2 >= 2)); };
        auto cells = [&]() { return (long long)a * b * (dim == 3 ? d : 1); };
        if (o.levels > 0) {
            for (int l = 1; l < o.levels; ++l) {
                if (!halvable()) {
                    delete h;
                    set_error("grid cannot be coarsened to the requested number of levels");
                    return BAH_ERR_ARG;
                }
                a /= 2; b /= 2; d /= 2; ++L;
            }
        } else {
            const int maxc = o.max_coarse_cells > 0 ? o.max_coarse_cells : 256;
            while (cells() > maxc && halvable()) {
                a /= 2; b /= 2; d /= 2; ++L;
            }
        }
        if (cells() > 4096) {
            delete h;
            set_error("coarsest level larger than 4096 cells; use more levels");
            return BAH_ERR_ARG;
        }
    }
    if (dim == 3 && L < 2) {
        delete h;
        set_error("3-D grids need at least 2 multigrid levels (the coarsest solve takes a Galerkin 27-point stencil)");
        return BAH_ERR_ARG;
    }
    c.L = L;
    c.alpha = o.shift_alpha >= 0.0 ? o.shift_alpha : (L < 5 ? kAlphaByLevels[L] : kAlphaDeep);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        set_error("cudaStreamCreate failed");
        return BAH_ERR_CUDA;
    }
    int s = dim == 3 ? build3(c, med, st) : build(c, med, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (s != BAH_OK) {
        delete h;
        return s;
    }
    *out = h;
    return BAH_OK;
}

void bah_destroy(bah_ctx* h) { delete h; }

int bah_sizes(const bah_ctx* h, long long* vector_len, int* levels) {
    if (!h) { set_error("ctx is NULL"); return BAH_ERR_ARG; }
    if (vector_len) *vector_len = (long long)h->c.vec_len();
    if (levels) *levels = h->c.L;
    return BAH_OK;
}

int bah_get_info(const bah_ctx* h, bah_info* out) {
    if (!h || !out) { set_error("bad argument"); return BAH_ERR_ARG; }
    const Ctx& c = h->c;
    out->levels = c.L;
    out->shift_alpha = c.alpha;
    out->coarse_points = c.dim == 3 ? c.d3[c.L - 1][0] * c.d3[c.L - 1][1] * c.d3[c.L - 1][2]
                                    : c.ln1[c.L - 1] * c.ln2[c.L - 1];
    out->cluster_level = c.sm_l0;
    out->cluster_ctas = c.sm_cs;
    out->cluster_smem_bytes = (long long)c.sm_bytes;
    out->block_iters = c.block_iters;
    out->block_failures = c.block_failures;
    return BAH_OK;
}

int bah_apply_operator(bah_ctx* h, const void* x, void* y, int nrhs, int conj, void* stream) {
    if (!h || !x || !y || nrhs < 0) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = c.vec_len();
    for (int k = 0; k < nrhs; ++k)
        apply_h(c, (const double2*)x + k * n, 0, (double2*)y + k * n, 0, nullptr, 0, conj ? 1 : 0, 1, st);
    BAH_CUDA_TRY(cudaGetLastError());
    return BAH_OK;
}

int bah_apply_preconditioner(bah_ctx* h, const void* r, void* z, int nrhs, void* stream) {
    if (!h || !r || !z || nrhs < 0) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = c.vec_len();
    Batch one;
    c.exact_status = BAH_OK;
    for (int k = 0; k < nrhs; ++k) {
        const double2* rk = (const double2*)r + k * n;
        double2* zk = (double2*)z + k * n;
        if (c.mode == BAH_MIXED) {
            precond_any(c, rk, n, c.ztmp, n, one, st);
            launch_convert<float2, double2>((const float2*)c.ztmp, zk, n, st);
        } else {
            precond_any(c, rk, n, zk, n, one, st);
        }
    }
    BAH_CUDA_TRY(cudaGetLastError());
    if (c.exact_status != BAH_OK) {
        set_error("an exact block solve failed inside the preconditioner");
        return c.exact_status;
    }
    return BAH_OK;
}

int bah_spectral_radius(bah_ctx* h, const void* x0, int iters, double* history, double* rho, void* stream) {
    if (!h || !x0 || iters < 1 || !rho) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = c.vec_len();
    double2* x = c.X;
    double2* y = c.R;
    double2* z = c.W;
    double2* t = c.Bs;
    KS ks;
    Batch one;
    c.exact_status = BAH_OK;
    launch_norm2((const double2*)x0, n, c.dpart, c.nrm, 0, 1, ks, st);
    launch_scale_copy((const double2*)x0, c.nrm, 0, x, n, 0, 0, 1, ks, st);
    std::vector<double> hist(iters);
    for (int k = 0; k < iters; ++k) {
        apply_h(c, x, 0, y, 0, nullptr, 0, 0, 1, st);
        if (c.mode == BAH_MIXED) {
            precond_any(c, (const double2*)y, n, c.ztmp, n, one, st);
            launch_convert<float2, double2>((const float2*)c.ztmp, z, n, st);
        } else {
            precond_any(c, (const double2*)y, n, z, n, one, st);
        }
        launch_sub(x, z, t, n, st);
        launch_norm2(t, n, c.dpart, c.nrm, 0, 1, ks, st);
        launch_scale_copy(t, c.nrm, 0, x, n, 0, 0, 1, ks, st);
        BAH_CUDA_TRY(cudaGetLastError());
        BAH_CUDA_TRY(cudaMemcpyAsync(&hist[k], c.nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
        BAH_CUDA_TRY(cudaStreamSynchronize(st));
        if (c.exact_status != BAH_OK) {
            set_error("an exact block solve failed inside the preconditioner");
            return c.exact_status;
        }
        if (!std::isfinite(hist[k])) { set_error("non-finite value in the power method"); return BAH_ERR_NONFINITE; }
        if (hist[k] == 0.0) { iters = k + 1; break; }
    }
    const int q = std::max(1, iters / 4);
    double acc = 0.0;
    for (int k = iters - q; k < iters; ++k) acc += std::log(std::max(hist[k], 1e-300));
    *rho = std::exp(acc / q);
    if (history)
        for (int k = 0; k < iters; ++k) history[k] = hist[k];
    return BAH_OK;
}

int bah_spectral_radius_z(bah_ctx* h, const void* x0, int iters, double* history, double* rho, void* stream) {
    if (!h || !x0 || iters < 1 || !rho) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    if (!c.exact) {
        set_error("bah_spectral_radius_z needs exact block solves (a 2-D context with block_rtol > 0)");
        return BAH_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t np = c.np, n = c.vec_len();
    const double ihx = 1.0 / c.h1, ihz = 1.0 / c.h2;
    KS ks;
    double2* v = c.W;                   // pressure-lattice iterate (np)
    double2* zero = c.Bs;               // a zero padded vector (the r of s_u = r_u - B^T e)
    double2* Y = c.X;                   // [A_s^{-1} s_u ; 0]
    double2* Q = c.R;                   // H [y ; 0] = [A y ; B y]
    double2* ep = c.etp;                // H_p,s^{-1} v, then Xi y
    auto solve = [&](int b, const double2* s, double2* e) {
        return c.mode == BAH_MIXED ? block_solve<BAH_MIXED>(c, b, s, e, st) : block_solve<BAH_FP64>(c, b, s, e, st);
    };
    c.exact_status = BAH_OK;
    BAH_CUDA_TRY(cudaMemsetAsync(zero, 0, n * sizeof(double2), st));
    BAH_CUDA_TRY(cudaMemsetAsync(Y, 0, n * sizeof(double2), st));
    launch_norm2((const double2*)x0, np, c.dpart, c.nrm, 0, 1, ks, st);
    launch_scale_copy((const double2*)x0, c.nrm, 0, v, np, 0, 0, 1, ks, st);
    std::vector<double> hist(iters);
    for (int k = 0; k < iters; ++k) {
        TRY(solve(2, v, ep));                                                    // H_p,s^{-1} v
        launch_u_rhs<BAH_FP64, double2>(c.n1, c.n2, ihx, ihz, zero, ep, c.esu, c.esu + np, st, 1, RhsStride());
        TRY(solve(0, c.esu, Y));                                                 // -A_s^{-1} B^T H_p,s^{-1} v
        TRY(solve(1, c.esu + np, Y + np));
        apply_h(c, Y, 0, Q, 0, nullptr, 0, 0, 1, st);                            // [A y ; B y]
        launch_distributor<BAH_FP64, double2>(c.n1, c.n2, ihx, ihz, c.f5x, Q, ep, st, 1, RhsStride());   // B A y - A_p B y
        launch_norm2(ep, np, c.dpart, c.nrm, 0, 1, ks, st);
        launch_scale_copy(ep, c.nrm, 0, v, np, 0, 0, 1, ks, st);
        BAH_CUDA_TRY(cudaGetLastError());
        BAH_CUDA_TRY(cudaMemcpyAsync(&hist[k], c.nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
        BAH_CUDA_TRY(cudaStreamSynchronize(st));
        if (!std::isfinite(hist[k])) { set_error("non-finite value in the power method"); return BAH_ERR_NONFINITE; }
        if (hist[k] == 0.0) { iters = k + 1; break; }
    }
    const int q = std::max(1, iters / 4);
    double acc = 0.0;
    for (int k = iters - q; k < iters; ++k) acc += std::log(std::max(hist[k], 1e-300));
    *rho = std::exp(acc / q);
    if (history)
        for (int k = 0; k < iters; ++k) history[k] = hist[k];
    return BAH_OK;
}

int bah_block_cycle(bah_ctx* h, int block, const void* b, void* x, void* stream) {
    if (!h || !b || !x || block < 0 || block > h->c.dim) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t np = c.np;
    Batch one;
    if (c.dim == 3) {
        if (c.mode == BAH_MIXED) {
            launch_convert<double2, float2>((const double2*)b, (float2*)c.v3B[0][block], np, st);
            float2* xx[1] = {(float2*)c.ztmp};
            MG3<BAH_MIXED>::cycle(c, 0, block, 1, xx, true, st);
            launch_convert<float2, double2>((const float2*)c.ztmp, (double2*)x, np, st);
        } else {
            BAH_CUDA_TRY(cudaMemcpyAsync(c.v3B[0][block], b, np * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            double2* xx[1] = {(double2*)x};
            MG3<BAH_FP64>::cycle(c, 0, block, 1, xx, true, st);
        }
        BAH_CUDA_TRY(cudaGetLastError());
        return BAH_OK;
    }
    if (c.mode == BAH_MIXED) {
        launch_convert<double2, float2>((const double2*)b, (float2*)c.vB[0][block], np, st);
        float2* o[1] = {(float2*)c.ztmp};
        MG<BAH_MIXED>::cycle(c, 0, block, 1, o, np, one, st);
        launch_convert<float2, double2>((const float2*)c.ztmp, (double2*)x, np, st);
    } else {
        BAH_CUDA_TRY(cudaMemcpyAsync(c.vB[0][block], b, np * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        double2* o[1] = {(double2*)x};
        MG<BAH_FP64>::cycle(c, 0, block, 1, o, np, one, st);
    }
    BAH_CUDA_TRY(cudaGetLastError());
    return BAH_OK;
}

int bah_level_stencil(const bah_ctx* h, int block, int level, double* out, int* rx, int* rz, int* n1, int* n2) {
    if (!h || block < 0 || block > h->c.dim || level < 0 || level >= h->c.L) { set_error("bad argument"); return BAH_ERR_ARG; }
    if (h->c.dim == 3) { set_error("bah_level_stencil describes 2-D stencils only"); return BAH_ERR_UNSUPPORTED; }
    const StencilF64& s = h->c.s64[level][block];
    if (rx) *rx = s.rx;
    if (rz) *rz = s.rz;
    if (n1) *n1 = s.n1;
    if (n2) *n2 = s.n2;
    if (out) {
        const size_t cnt = (size_t)(2 * s.rx + 1) * (2 * s.rz + 1) * s.n1 * s.n2;
        BAH_CUDA_TRY(cudaMemcpy(out, s.S, cnt * sizeof(double2), cudaMemcpyDeviceToHost));
    }
    return BAH_OK;
}

int bah_profile_control(bah_ctx* h, unsigned mask, int reset) {
    if (!h) { set_error("ctx is NULL"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    prof_flush(c);
    c.tmask = mask;
    if (reset) {
        c.launches = 0;
        for (int k = 0; k < 16; ++k) { c.cls_launch[k] = 0; c.cls_calls[k] = 0; c.cls_ms[k] = 0; c.cls_bytes[k] = 0; }
    }
    return BAH_OK;
}

int bah_profile_read(bah_ctx* h, bah_profile* out) {
    if (!h || !out) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    prof_flush(c);
    out->launches = c.launches;
    for (int k = 0; k < 16; ++k) {
        out->class_launches[k] = c.cls_launch[k];
        out->class_calls[k] = c.cls_calls[k];
        out->class_ms[k] = c.cls_ms[k];
        out->class_bytes[k] = c.cls_bytes[k];
    }
    return BAH_OK;
}

}  // extern "C"

// H x = b (adjoint = 0) or H^H x = b, i.e. H conj(x) = conj(b) (adjoint = 1)
static int solve_impl(bah_ctx* h, const void* b, void* x, int nrhs, double rtol, bah_stats* stats, void* stream,
                      int adjoint) {
    if (!h || !b || !x || nrhs < 0 || !(rtol > 0.0)) { set_error("bad argument"); return BAH_ERR_ARG; }
    NvtxRange nv(adjoint ? "bah_solve_adjoint" : "bah_solve");
    Ctx& c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = c.vec_len();
    const bool dev_b = is_device_ptr(b), dev_x = is_device_ptr(x);
    if (dev_b != dev_x) { set_error("b and x must both be device or both be host pointers"); return BAH_ERR_ARG; }
    int first_fail = BAH_OK;
    c.exact_status = BAH_OK;
    for (int k0 = 0; k0 < nrhs; k0 += c.nbatch) {
        const int nr = std::min(c.nbatch, nrhs - k0);
        const double2* bk = (const double2*)b + (size_t)k0 * n;
        double2* xk = (double2*)x + (size_t)k0 * n;
        BAH_CUDA_TRY(cudaMemcpyAsync(c.Bs, bk, (size_t)nr * n * sizeof(double2),
                                     dev_b ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        {
            Prof pr(c, BAH_K_SMALL, st, (double)nr * c.np * 32.0);
            if (c.dim == 3) launch_sanitize3(c.Bs, c.n1, c.n2, c.n3, nr, st);
            else launch_sanitize(c.Bs, c.n1, c.n2, nr, st);
            if (adjoint) launch_conj(c.Bs, (size_t)nr * n, st);
        }
        double2* xd = dev_x ? xk : c.X;
        int s = c.o.block_krylov ? fgmres_block(c, c.Bs, xd, nr, rtol, stats ? stats + k0 : nullptr, st)
                                 : fgmres_batch(c, c.Bs, xd, nr, rtol, stats ? stats + k0 : nullptr, st);
        if (s == BAH_ERR_CUDA || s == BAH_ERR_OOM || s == BAH_ERR_ARG) return s;
        if (adjoint) {
            Prof pr(c, BAH_K_SMALL, st, (double)nr * n * 32.0);
            launch_conj(xd, (size_t)nr * n, st);
        }
        if (!dev_x)
            BAH_CUDA_TRY(cudaMemcpyAsync(xk, c.X, (size_t)nr * n * sizeof(double2), cudaMemcpyDeviceToHost, st));
        if (s != BAH_OK && first_fail == BAH_OK) first_fail = s;
    }
    BAH_CUDA_TRY(cudaStreamSynchronize(st));
    return first_fail;
}

extern "C" {

int bah_solve(bah_ctx* h, const void* b, void* x, int nrhs, double rtol, bah_stats* stats, void* stream) {
    return solve_impl(h, b, x, nrhs, rtol, stats, stream, 0);
}

int bah_solve_adjoint(bah_ctx* h, const void* b, void* y, int nrhs, double rtol, bah_stats* stats, void* stream) {
    return solve_impl(h, b, y, nrhs, rtol, stats, stream, 1);
}

int bah_misfit(bah_ctx* h, const void* x, const void* d, const int* rec, int nrec, int nrhs, void* adj,
               double* misfit, void* stream) {
    if (!h || !x || !d || !rec || !adj || !misfit || nrec < 1 || nrhs < 0) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = c.vec_len();
    BAH_CUDA_TRY(cudaMemsetAsync(adj, 0, (size_t)nrhs * n * sizeof(double2), st));
    if (nrhs == 0) return BAH_OK;
    launch_misfit((const double2*)x, (const double2*)d, rec, nrec, nrhs, n, (double2*)adj, misfit, st);
    BAH_CUDA_TRY(cudaGetLastError());
    return BAH_OK;
}

int bah_gradient(bah_ctx* h, const void* x_fwd, const void* y_adj, int nrhs, double* g_lambda, double* g_mu,
                 double* g_rho, void* stream) {
    if (!h || !x_fwd || !y_adj || !g_lambda || !g_mu || !g_rho || nrhs < 0) { set_error("bad argument"); return BAH_ERR_ARG; }
    Ctx& c = h->c;
    if (c.dim == 3) { set_error("the adjoint gradient is implemented for 2-D grids"); return BAH_ERR_UNSUPPORTED; }
    if (nrhs == 0) return BAH_OK;
    launch_gradient(c.n1, c.n2, c.h1, c.h2, c.omega, c.cinv, c.gam, c.vec_len(), nrhs, (const double2*)x_fwd,
                    (const double2*)y_adj, g_lambda, g_mu, g_rho, (cudaStream_t)stream);
    BAH_CUDA_TRY(cudaGetLastError());
    return BAH_OK;
}

}  // extern "C"
