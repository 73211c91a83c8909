// C-ABI entry points of libxk: context, input loading, workspace layout,
// host-side index structures, and the enqueueing of the implicit step.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "xk_bcr.cuh"
#include "xk_gmres.cuh"
#include "xk_internal.cuh"

using namespace xk;

// A chunk of controlled steps captured once and replayed with one graph launch.
struct StepGraph {
    int steps = 0;
    bool ctl_copy = false;           // ends with the copy of the control block to its host mirror
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;           // kernel nodes of one replay
};

struct xk_ctx {
    xk_config cfg;
    cudaStream_t st = nullptr;
    std::string err;
    // host copies of the inputs
    int S = 0, E = 0, R = 0, L = 0, W = 0, Rph = 0;
    std::vector<int> elem, rtype, reac, prod, form, prow;
    std::vector<double> mass, arr, troe, nasa, lam, dlam, J0, sigma, sigma_abs, P, T, Kzz, dcoef;
    double mu = 0.5, tf = 0.5, g = 0, mbar = 0, alpha_T = 0;
    std::vector<double> sigma_s;   // Rayleigh cross sections S x W (empty: none)
    double albedo = 0.0;
    int diffuse = 0;
    bool have_net = false, have_photo = false, have_atm = false;
    bool rates_valid = false;      // k_f, k_r of the loaded network and atmosphere are in the workspace
    // host index structures
    std::vector<int> yp, yent, jp, jcol, jtp, jrs, jdq, abs_sp;
    std::vector<int> pg_p, pg_v, pg_s, pg_code;   // reaction graph of the pathway analyser
    std::vector<int> eq_sp, eq_se, eq_ep, eq_ey, eq_eij;   // sparse element structure (equilibrium)
    std::vector<double> eq_sc, eq_ec;
    std::vector<double> sig_abs_c;
    std::vector<int> sca_sp;           // species with a non-zero scattering cross section
    std::vector<double> sig_sca_c;
    // device
    char *ws = nullptr;
    size_t ws_bytes = 0;
    Col col{};
    Ctl *ctl = nullptr, *ctl_aux = nullptr;
    Ctl *ctl_host = nullptr;   // pinned
    double *A64 = nullptr, *lo64 = nullptr, *up64 = nullptr;
    float *A32 = nullptr, *lo32 = nullptr, *up32 = nullptr;
    int *ridx = nullptr, *sig = nullptr, *pinfo = nullptr;
    int *ridx32 = nullptr, *sig32 = nullptr;   // row/column pivots of the FP32 inversion
    double *dinv = nullptr;                    // FP64 factorization: LU factors of the current panel's pivot block
    double *ymid = nullptr;                    // twisted sweeps: the two products that meet at the middle layer
    unsigned *bar = nullptr;
    double *gsol = nullptr;
    // FGMRES buffers
    double *V = nullptr, *Z = nullptr, *gw = nullptr, *h1 = nullptr, *h2 = nullptr, *red = nullptr, *partials = nullptr;
    double *rowd = nullptr, *bhat = nullptr;   // row equilibration: diagonal of I/dt - J, scaled right-hand side
    float *gbuf = nullptr;                       // panel buffer of the FP32 inversion without pivoting
    double *s64 = nullptr, *pin = nullptr, *pout = nullptr;   // scaling of the reused FP64 factorization
    unsigned *counter = nullptr;
    GmState *gm = nullptr;
    FactorPlan plan{};     // plan of the context's precision
    FactorPlan plan64{};   // FP64 plan (fallback of the mixed path)
    ClusterPlan cplan{};   // cluster-resident FP32 inversion (mixed path, no pivoting)
    bool use_cluster = false;
    SolvePlan splan{};     // sweeps with those inverses on one cluster
    bool use_cluster_solve = false;
    SolvePlan splan64{};   // sweeps with the pivoted FP64 inverses on one cluster
    bool use_cluster_solve64 = false;
    BcrPlan bcr;           // block cyclic reduction on the tensor cores (mixed path, fp32_bcr)
    bool use_bcr = false;
    bool ready = false;
    // equilibrium initial state and pathway analyser
    PathGraph pgraph{};
    EqIndex eqix{};
    int *eq_iters = nullptr, *eq_status = nullptr, *path_src = nullptr;
    double *path_w = nullptr;   // [L][R][2] edge weights of the pathway search
    // variable-order BDF: history buffers [kBdfHist][L][S], predictor, history terms, new state, step
    double *bdfY = nullptr, *bdf_yhat = nullptr, *bdf_g = nullptr, *bdf_ynew = nullptr, *bdf_delta = nullptr;
    BdfResult *bdf_res = nullptr;
    // Lagrangian parcel scheme: its buffers in the workspace (ParcelArgs without the policy)
    ParcelArgs parcel{};
    double *parcel_kzz0 = nullptr;   // [L] zero eddy profile: the molecular part of u, v
    ParcelState *parcel_host = nullptr;   // pinned
    int parcel_max_visit = 0;
    // captured chunks of controlled steps (cfg.use_graphs), dropped whenever a plan, the workspace
    // or the batch slot changes
    std::vector<StepGraph> graphs;
    cudaStream_t cap_st = nullptr;   // capture stream (the legacy default stream cannot be captured)
    // tracing
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[XK_PH_COUNT];
    size_t ev_used[XK_PH_COUNT] = {};
};

namespace {

constexpr size_t kMaxEventPairs = 65536;

// Marks one phase of a step with a pair of CUDA events when tracing is on.
struct PhaseMark {
    xk_ctx *c;
    int ph;
    cudaEvent_t end = nullptr;
    PhaseMark(xk_ctx *ctx, int phase) : c(ctx), ph(phase)
    {
        if (!c->prof || c->ev_used[ph] >= kMaxEventPairs) return;
        auto &v = c->ev[ph];
        if (c->ev_used[ph] == v.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            v.push_back({a, b});
        }
        auto &pr = v[c->ev_used[ph]++];
        cudaEventRecord(pr.first, c->st);
        end = pr.second;
    }
    ~PhaseMark()
    {
        if (end) cudaEventRecord(end, c->st);
    }
};

int fail(xk_ctx *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(xk_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_check(xk_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "%s: %s", where, cudaGetErrorString(e));
    return XK_OK;
}

Policy policy_of(const xk_config &c)
{
    Policy p;
    p.dt_max = c.dt_max; p.rel_reject = c.rel_reject; p.rel_target = c.rel_target;
    p.grow_max = c.grow_max; p.shrink_min = c.shrink_min; p.neg_tol = c.neg_tol;
    p.f_floor = c.f_floor; p.dt_min = c.dt_min; p.ss_dt = c.ss_dt; p.ss_tol = c.ss_tol;
    return p;
}

struct Bump {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Index structures built once per network (symbolic, no arithmetic of the method).
void build_indices(xk_ctx *c)
{
    const int S = c->S, R = c->R;
    // species-major stoichiometry, in reaction order: for r, for slot s: reactant, then product
    std::vector<std::vector<int>> ys(S);
    for (int r = 0; r < R; ++r)
        for (int s = 0; s < 3; ++s) {
            int i = c->reac[3 * r + s];
            if (i >= 0) ys[i].push_back(r * 16 + (-1 + 8));
            int j = c->prod[3 * r + s];
            if (j >= 0) ys[j].push_back(r * 16 + (1 + 8));
        }
    c->yp.assign(S + 1, 0);
    c->yent.clear();
    for (int y = 0; y < S; ++y) {
        c->yent.insert(c->yent.end(), ys[y].begin(), ys[y].end());
        c->yp[y + 1] = (int)c->yent.size();
    }
    // Jacobian rows: for r, side, slot s (column j), then each reactant (+) / product (-) row
    std::vector<std::vector<std::pair<int, int>>> rows(S);
    for (int r = 0; r < R; ++r)
        for (int side = 0; side < 2; ++side)
            for (int s = 0; s < 3; ++s) {
                int j = side == 0 ? c->reac[3 * r + s] : c->prod[3 * r + s];
                if (j < 0) continue;
                int rs = r * 8 + side * 3 + s;
                for (int q = 0; q < 3; ++q) {
                    int i = c->reac[3 * r + q];
                    if (i >= 0) rows[i].push_back({j | (1 << 16), rs});
                    int k = c->prod[3 * r + q];
                    if (k >= 0) rows[k].push_back({j, rs});
                }
            }
    // grouped by column: row i's distinct columns jcol[jp[i] .. jp[i+1]) in increasing order, each
    // with its terms jrs[jtp[q] .. jtp[q+1]) in reaction order, a term being (slot << 1) | (reactant
    // row: +d, product row: -d); jdq[i] is the entry of column i in row i (-1 if none)
    c->jp.assign(S + 1, 0);
    c->jcol.clear();
    c->jtp.assign(1, 0);
    c->jrs.clear();
    c->jdq.assign(S, -1);
    for (int i = 0; i < S; ++i) {
        std::vector<std::pair<int, int>> ent = rows[i];
        std::stable_sort(ent.begin(), ent.end(),
                         [](const std::pair<int, int> &a, const std::pair<int, int> &b) {
                             return (a.first & 0xffff) < (b.first & 0xffff);
                         });
        for (size_t e = 0; e < ent.size(); ++e) {
            const int j = ent[e].first & 0xffff;
            if (e == 0 || j != (ent[e - 1].first & 0xffff)) {
                if (e > 0) c->jtp.push_back((int)c->jrs.size());
                if (j == i) c->jdq[i] = (int)c->jcol.size();
                c->jcol.push_back(j);
            }
            c->jrs.push_back((ent[e].second << 1) | ((ent[e].first >> 16) > 0 ? 1 : 0));
        }
        if (!ent.empty()) c->jtp.push_back((int)c->jrs.size());
        c->jp[i + 1] = (int)c->jcol.size();
    }
    // absorbers with a non-zero cross section somewhere
    c->abs_sp.clear();
    c->sig_abs_c.clear();
    if (c->have_photo && c->W > 0)
        for (int y = 0; y < S; ++y) {
            bool nz = false;
            for (int w = 0; w < c->W; ++w) nz |= c->sigma_abs[(size_t)y * c->W + w] != 0.0;
            if (!nz) continue;
            c->abs_sp.push_back(y);
            c->sig_abs_c.insert(c->sig_abs_c.end(), c->sigma_abs.begin() + (size_t)y * c->W,
                                c->sigma_abs.begin() + (size_t)(y + 1) * c->W);
        }
    // scatterers with a non-zero cross section somewhere
    c->sca_sp.clear();
    c->sig_sca_c.clear();
    if (c->have_photo && c->W > 0 && !c->sigma_s.empty())
        for (int y = 0; y < S; ++y) {
            bool nz = false;
            for (int w = 0; w < c->W; ++w) nz |= c->sigma_s[(size_t)y * c->W + w] != 0.0;
            if (!nz) continue;
            c->sca_sp.push_back(y);
            c->sig_sca_c.insert(c->sig_sca_c.end(), c->sigma_s.begin() + (size_t)y * c->W,
                                c->sigma_s.begin() + (size_t)(y + 1) * c->W);
        }
    // equilibrium: each species' elements, and each Newton-system entry's species (increasing)
    const int E = c->E;
    c->eq_sp.assign(S + 1, 0);
    c->eq_se.clear();
    c->eq_sc.clear();
    for (int y = 0; y < S; ++y) {
        for (int e = 0; e < E; ++e)
            if (c->elem[(size_t)y * E + e] != 0) {
                c->eq_se.push_back(e);
                c->eq_sc.push_back((double)c->elem[(size_t)y * E + e]);
            }
        c->eq_sp[y + 1] = (int)c->eq_se.size();
    }
    c->eq_ep.assign(1, 0);
    c->eq_ey.clear();
    c->eq_ec.clear();
    c->eq_eij.clear();
    auto add_entry = [&](int code, int i, int j) {
        for (int y = 0; y < S; ++y) {
            const double ai = c->elem[(size_t)y * E + i], aj = j >= 0 ? c->elem[(size_t)y * E + j] : 1.0;
            if (ai != 0.0 && aj != 0.0) {
                c->eq_ey.push_back(y);
                c->eq_ec.push_back(ai * aj);
            }
        }
        c->eq_eij.push_back(code);
        c->eq_ep.push_back((int)c->eq_ey.size());
    };
    if (E <= 30) {
        for (int i = 0; i < E; ++i)
            for (int j = i; j < E; ++j) add_entry(i * 32 + j, i, j);
        for (int i = 0; i < E; ++i) add_entry(-1 - i, i, -1);
    }
    // pathway graph: each reaction direction gives an edge from every species it consumes to every
    // species it produces (itself excepted), grouped by source, then target, codes increasing
    std::vector<std::vector<std::pair<int, int>>> out(S);   // (target, code) per source
    for (int r = 0; r < R; ++r)
        for (int dir = 0; dir < 2; ++dir) {
            const int *frm = dir == 0 ? &c->reac[3 * r] : &c->prod[3 * r];
            const int *to = dir == 0 ? &c->prod[3 * r] : &c->reac[3 * r];
            for (int a = 0; a < 3; ++a) {
                const int u = frm[a];
                if (u < 0 || (a > 0 && frm[0] == u) || (a > 1 && frm[1] == u)) continue;
                for (int t = 0; t < 3; ++t) {
                    const int v = to[t];
                    if (v < 0 || v == u || (t > 0 && to[0] == v) || (t > 1 && to[1] == v)) continue;
                    out[u].push_back({v, 2 * r + dir});
                }
            }
        }
    c->pg_p.assign(S + 1, 0);
    c->pg_v.clear();
    c->pg_s.assign(1, 0);
    c->pg_code.clear();
    for (int u = 0; u < S; ++u) {
        auto &ev = out[u];
        std::stable_sort(ev.begin(), ev.end(),
                         [](const std::pair<int, int> &a, const std::pair<int, int> &b) { return a.first < b.first; });
        for (size_t i = 0; i < ev.size(); ++i) {
            if (i == 0 || ev[i].first != ev[i - 1].first) {
                if (i > 0) c->pg_s.push_back((int)c->pg_code.size());
                c->pg_v.push_back(ev[i].first);
            }
            c->pg_code.push_back(ev[i].second);
        }
        if (!ev.empty()) c->pg_s.push_back((int)c->pg_code.size());
        c->pg_p[u + 1] = (int)c->pg_v.size();
    }
}

// Krylov basis size: FGMRES(m) of the mixed path; in FP64 mode only the refinement around the
// FP64 factorization runs, with at most refine_max_iter iterations.
int basis_size(const xk_ctx *c)
{
    int m = std::min(std::max(c->cfg.gmres_restart, 1), kMaxBasis);
    if (c->cfg.precision == XK_PREC_FP64) m = std::min(m, std::max(c->cfg.refine_max_iter, 1));
    return m;
}

// Lay out the workspace; with base == nullptr only the size is computed.
size_t layout(xk_ctx *c, char *base)
{
    Bump b{base};
    const int S = c->S, R = c->R, L = c->L, W = c->W, Rph = c->Rph;
    const int Sabs = (int)c->abs_sp.size();
    const size_t LS = (size_t)L * S, LR = (size_t)L * R;
    const int ld = round_up(S, 32);
    Col &k = c->col;
    Col t{};
    t.S = S; t.E = c->E; t.R = R; t.L = L; t.W = W; t.Rph = Rph; t.Sabs = Sabs; t.ld = ld;
    t.elem = b.take<int>(std::max<size_t>(1, (size_t)S * c->E));
    t.mass = b.take<double>(S); t.nasa = b.take<double>(15 * (size_t)S); t.dcoef = b.take<double>(S);
    t.arr = b.take<double>(9 * (size_t)R); t.troe = b.take<double>(4 * (size_t)R);
    t.rtype = b.take<int>(R); t.reac = b.take<int>(3 * (size_t)R); t.prod = b.take<int>(3 * (size_t)R);
    t.form = b.take<int>(R); t.prow = b.take<int>(R);
    t.yp = b.take<int>(S + 1); t.yent = b.take<int>(std::max<size_t>(1, c->yent.size()));
    t.jp = b.take<int>(S + 1); t.jcol = b.take<int>(std::max<size_t>(1, c->jcol.size()));
    t.jtp = b.take<int>(std::max<size_t>(1, c->jtp.size()));
    t.jrs = b.take<int>(std::max<size_t>(1, c->jrs.size()));
    t.jdq = b.take<int>(S);
    t.J0 = b.take<double>(std::max(W, 1)); t.dlam = b.take<double>(std::max(W, 1));
    t.sigma = b.take<double>(std::max<size_t>(1, (size_t)Rph * W));
    t.sig_abs = b.take<double>(std::max<size_t>(1, (size_t)Sabs * W));
    t.abs_sp = b.take<int>(std::max(Sabs, 1));
    t.mu = c->mu; t.tf = c->tf;
    const int Ssca = (int)c->sca_sp.size();
    t.Ssca = Ssca;
    t.diffuse = (c->diffuse && W > 0) ? 1 : 0;
    t.albedo = c->albedo;
    t.sig_sca = b.take<double>(std::max<size_t>(1, (size_t)Ssca * W));
    t.sca_sp = b.take<int>(std::max(Ssca, 1));
    t.alpha_s = b.take<double>((size_t)L * std::max(W, 1));
    t.rt = b.take<double>(t.diffuse ? 4 * (size_t)L * W : 1);
    t.photo_jac = (c->cfg.photo_jacobian && W > 0 && Rph > 0) ? 1 : 0;
    t.pbeta = b.take<double>(t.photo_jac ? (size_t)L * W : 1);
    t.pdJ = b.take<double>(t.photo_jac ? (size_t)L * W : 1);
    t.pdk = b.take<double>(t.photo_jac ? (size_t)L * Rph : 1);
    t.P = b.take<double>(L); t.T = b.take<double>(L); t.Kzz = b.take<double>(L);
    t.g = c->g; t.mbar = c->mbar; t.alpha_T = c->alpha_T;
    t.ngas = b.take<double>(L); t.z = b.take<double>(L); t.dz = b.take<double>(L); t.dzi = b.take<double>(L);
    t.u = b.take<double>(std::max<size_t>(1, (size_t)(L - 1) * S));
    t.v = b.take<double>(std::max<size_t>(1, (size_t)(L - 1) * S));
    t.tdg = b.take<double>(LS); t.tlo = b.take<double>(LS); t.tup = b.take<double>(LS); t.rs = b.take<double>(LS);
    t.grt = b.take<double>(LS); t.lnkc = b.take<double>(LR);
    t.kf = b.take<double>(LR); t.kr = b.take<double>(LR);
    t.kph = b.take<double>((size_t)L * std::max(Rph, 1));
    t.alpha = b.take<double>((size_t)L * std::max(W, 1)); t.Jw = b.take<double>((size_t)L * std::max(W, 1));
    t.w = b.take<double>(LR); t.d = b.take<double>(6 * LR); t.dw = b.take<double>(LR);
    t.n = b.take<double>(LS); t.F = b.take<double>(LS); t.s = b.take<double>(LS); t.b = b.take<double>(LS);
    t.x = b.take<double>(LS); t.delta = b.take<double>(LS); t.tmp = b.take<double>(LS);
    k = t;
    c->gsol = b.take<double>(LS);
    // FP64 blocks in both modes: the mixed path falls back to them when the
    // FP32-preconditioned solve does not converge
    c->A64 = b.take<double>((size_t)L * S * ld);
    c->lo64 = b.take<double>(LS);
    c->up64 = b.take<double>(LS);
    // FGMRES: around the FP32 inversion (mixed), around FP64 factorizations (both modes)
    const int m = basis_size(c);
    c->V = b.take<double>((size_t)(m + 1) * LS);
    c->Z = b.take<double>((size_t)m * LS);
    c->gw = b.take<double>(LS);
    c->rowd = b.take<double>(LS);
    c->bhat = b.take<double>(LS);
    c->h1 = b.take<double>(kMaxBasis + 1);
    c->h2 = b.take<double>(kMaxBasis + 1);
    c->red = b.take<double>(8);
    c->partials = b.take<double>((size_t)kGmPartialBlocks * (kMaxBasis + 1));
    c->counter = b.take<unsigned>(8);
    c->gm = b.take<GmState>(1);
    if (c->cfg.precision == XK_PREC_FP64) {
        c->A32 = nullptr; c->lo32 = nullptr; c->up32 = nullptr;
    } else if (c->cfg.fp32_bcr) {
        // FP32 blocks padded to Sp x Sp per layer (identity in the padding), and the reduction's arrays
        const BcrSizes z = bcr_sizes(L, S);
        BcrPlan &q = c->bcr;
        c->A32 = b.take<float>(z.floats_D);
        c->lo32 = b.take<float>(LS);
        c->up32 = b.take<float>(LS);
        q.D = c->A32; q.lo = c->lo32; q.up = c->up32;
        q.INV = b.take<float>(z.floats_INV);
        q.TMP = b.take<float>(z.floats_TMP);
        q.CP = b.take<float>(z.floats_CP);
        q.PQ = b.take<float>(z.floats_PQ);
        q.bw = b.take<float>(z.floats_vec);
        q.tw = b.take<float>(z.floats_vec);
        q.xw = b.take<float>(z.floats_vec);
        q.gemm_d = b.take<TcTask>(std::max(z.ngemm, 1));
        q.leaf_d = b.take<BcrLeaf>(std::max(z.nleaf, 1));
        q.mv_d = b.take<BcrMv>(std::max(z.nmv, 1));
        q.maps_d = b.take<CUtensorMap>(10);
        q.l0_d = b.take<int>(L);
        q.sol_d = b.take<BcrStage>(std::max(z.nsol, 1));
        c->gbuf = nullptr;
        c->s64 = b.take<double>(LS);
        c->pin = b.take<double>(LS);
        c->pout = b.take<double>(LS);
        c->ridx32 = b.take<int>(LS);
        c->sig32 = b.take<int>(LS);
    } else {
        c->A32 = b.take<float>((size_t)L * S * ld);
        c->lo32 = b.take<float>(LS);
        c->up32 = b.take<float>(LS);
        c->gbuf = b.take<float>(4 * (size_t)S * 32);
        c->s64 = b.take<double>(LS);
        c->pin = b.take<double>(LS);
        c->pout = b.take<double>(LS);
        c->ridx32 = b.take<int>(LS);    // the FP64 factorization's pivots stay intact for reuse
        c->sig32 = b.take<int>(LS);
    }
    c->ridx = b.take<int>(LS);
    c->sig = b.take<int>(LS);
    c->pinfo = b.take<int>(1 + 4 * 64);
    c->dinv = b.take<double>(32 * 32);
    c->ymid = b.take<double>(2 * (size_t)S);
    c->bar = b.take<unsigned>(8);
    c->bcr.bar = c->bar ? c->bar + 4 : nullptr;      // words 4-5: the reduction's solve
    c->ctl = b.take<Ctl>(1);
    c->ctl_aux = b.take<Ctl>(1);
    // Lagrangian parcel scheme
    ParcelArgs &q = c->parcel;
    q.N = k.n;
    q.Nold = b.take<double>(LS);
    const size_t ifc = std::max<size_t>(1, (size_t)(L - 1) * S);
    q.um = b.take<double>(ifc);
    q.vm = b.take<double>(ifc);
    q.A = b.take<double>(2 * (size_t)S * S);
    q.vmr = b.take<double>(S);
    q.w = b.take<double>(std::max(R, 1));
    q.dd = b.take<double>(6 * (size_t)std::max(R, 1));
    q.st = b.take<ParcelState>(1);
    c->parcel_kzz0 = b.take<double>(L);
    // equilibrium initial state and pathway analyser
    c->eq_iters = b.take<int>(L);
    c->eq_status = b.take<int>(L);
    c->path_src = b.take<int>(std::max(S, 1));
    c->path_w = b.take<double>(std::max<size_t>(1, 2 * LR));
    c->bdfY = b.take<double>(kBdfHist * LS);
    c->bdf_yhat = b.take<double>(LS);
    c->bdf_g = b.take<double>(LS);
    c->bdf_ynew = b.take<double>(LS);
    c->bdf_delta = b.take<double>(LS);
    c->bdf_res = b.take<BdfResult>(1);
    EqIndex &ei = c->eqix;
    ei.sp = b.take<int>(S + 1);
    ei.se = b.take<int>(std::max<size_t>(1, c->eq_se.size()));
    ei.sc = b.take<double>(std::max<size_t>(1, c->eq_sc.size()));
    ei.ep = b.take<int>(c->eq_ep.size());
    ei.ey = b.take<int>(std::max<size_t>(1, c->eq_ey.size()));
    ei.ec = b.take<double>(std::max<size_t>(1, c->eq_ec.size()));
    ei.eij = b.take<int>(std::max<size_t>(1, c->eq_eij.size()));
    ei.nent = (int)c->eq_eij.size();
    c->pgraph.gp = b.take<int>(S + 1);
    c->pgraph.gv = b.take<int>(std::max<size_t>(1, c->pg_v.size()));
    c->pgraph.gs = b.take<int>(std::max<size_t>(1, c->pg_s.size()));
    c->pgraph.gcode = b.take<int>(std::max<size_t>(1, c->pg_code.size()));
    return b.off + 256;
}

template <typename T>
void up(xk_ctx *c, const T *dst, const std::vector<T> &v)
{
    if (!v.empty()) cudaMemcpyAsync((void *)dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->st);
}

BlockSys<double> sys64(xk_ctx *c)
{
    BlockSys<double> s;
    s.D = c->A64; s.lo = c->lo64; s.up = c->up64; s.perm = c->ridx; s.iperm = c->sig;
    s.pinfo = c->pinfo; s.bar = c->bar; s.L = c->L; s.S = c->S; s.ld = c->col.ld;
    return s;
}

BlockSys<float> sys32(xk_ctx *c)
{
    BlockSys<float> s;
    s.D = c->A32; s.lo = c->lo32; s.up = c->up32; s.perm = c->ridx32; s.iperm = c->sig32;
    s.pinfo = c->pinfo; s.bar = c->bar; s.L = c->L; s.S = c->S; s.ld = c->col.ld;
    return s;
}

// Event marks around the reduction's product and leaf launches (tracing).
struct StageMarks : BcrTimer {
    xk_ctx *c;
    PhaseMark *open = nullptr;
    explicit StageMarks(xk_ctx *ctx) : c(ctx) {}
    void begin(int kind) override { open = new PhaseMark(c, kind == kBcrGemm ? XK_PH_TC : XK_PH_LEAF); }
    void end(int) override
    {
        delete open;
        open = nullptr;
    }
};

// FP32 block inversions of the mixed path
cudaError_t factor32(xk_ctx *c, Ctl *ctl, const int *skip)
{
    if (c->use_bcr) {
        if (!c->prof) return bcr_factor(c->bcr, skip, ctl, c->st);
        StageMarks marks(c);
        return bcr_factor(c->bcr, skip, ctl, c->st, &marks);
    }
    if (c->cfg.fp32_pivoting) return launch_factor<float>(sys32(c), c->plan, ctl, c->st, skip);
    if (c->use_cluster) return launch_factor_cluster(sys32(c), c->cplan, c->gbuf, ctl, c->st, skip);
    return launch_factor_nopivot(sys32(c), c->plan, c->gbuf, ctl, c->st, skip);
}

// sweeps with the FP32 inverses
cudaError_t solve32(xk_ctx *c, const double *b, double *x, Ctl *ctl, cudaStream_t st, const double *bscale,
                    const int *skip)
{
    if (c->use_bcr) return bcr_solve(c->bcr, b, x, bscale, nullptr, skip, ctl, st);
    if (c->use_cluster_solve && c->use_cluster && cluster_twisted(c->cplan, c->L) && c->splan.twisted)
        return launch_solve_twisted<float>(sys32(c), c->splan, false, b, x, c->gsol, c->ymid, ctl, st, bscale, skip);
    if (c->use_cluster_solve && !(c->use_cluster && cluster_twisted(c->cplan, c->L)))
        return launch_solve_cluster<float>(sys32(c), c->splan, false, b, x, c->gsol, ctl, st, bscale, skip);
    return launch_solve<float>(sys32(c), c->plan, b, x, c->gsol, ctl, st, bscale, skip);
}

// sweeps with the (pivoted) FP64 inverses
cudaError_t solve64(xk_ctx *c, const FactorPlan &plan, const double *b, double *x, Ctl *ctl, cudaStream_t st,
                    const double *bscale, const int *skip, const double *xscale)
{
    if (c->use_cluster_solve64 && plan.twisted && c->L >= 3 && plan.ctas >= 2)
        return launch_solve_twisted<double>(sys64(c), c->splan64, true, b, x, c->gsol, c->ymid, ctl, st, bscale, skip,
                                            xscale);
    if (c->use_cluster_solve64)
        return launch_solve_cluster<double>(sys64(c), c->splan64, true, b, x, c->gsol, ctl, st, bscale, skip, xscale);
    return launch_solve<double>(sys64(c), plan, b, x, c->gsol, ctl, st, bscale, skip, xscale);
}

// FP64 plans: column-by-column panel factorization (k_factor), or each panel's pivots chosen
// first (k_factor_pv) when the context asks for it
void set_preview(xk_ctx *c, FactorPlan *p)
{
    p->preview = c->cfg.fp64_panel ? 1 : 0;
    p->dinv = c->dinv;
    // both ends at once (column-by-column kernel) when the sweeps can follow on two clusters
    p->twisted = (c->cfg.twisted && !p->preview && c->use_cluster_solve64 && c->splan64.twisted) ? 1 : 0;
}

// A control block with nothing decided yet and the context's bound on device-side waits.
Ctl fresh_ctl(const xk_ctx *c)
{
    Ctl init{};
    init.wait_polls = c->cfg.wait_polls > 0 ? (unsigned long long)c->cfg.wait_polls : 0ull;
    return init;
}

// A bounded wait gave up: the barrier words hold arrivals of the abandoned launch, so clear them
// (and the flag) before the context is used again.
int timed_out(xk_ctx *c)
{
    cudaMemsetAsync(c->bar, 0, 8 * sizeof(unsigned), c->st);
    cudaMemsetAsync(&c->ctl->err_timeout, 0, sizeof(int), c->st);
    cudaMemsetAsync(&c->ctl_aux->err_timeout, 0, sizeof(int), c->st);
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "clearing a timed-out wait: %s", cudaGetErrorString(e));
    return fail(c, XK_ETIMEOUT, "a device-side wait timed out");
}

int need_ready(xk_ctx *c)
{
    if (!c) return XK_EINVAL;
    if (!c->ready) return fail(c, XK_EINVAL, "workspace not set (load network, photolysis and atmosphere, then xk_set_workspace)");
    cudaSetDevice(c->cfg.device);
    return XK_OK;
}

// FGMRES in FP64 on the exact operator, preconditioned by a fresh FP64 factorization (the plain FP64
// path, and the mixed path's FP64 route): the right-hand side and residuals are row-equilibrated by
// c->rowd, which the preconditioner undoes before applying the stored inverses.
void enqueue_refine64(xk_ctx *c, const Col &col, Ctl *ctl, const FactorPlan &plan, const int *skip, int max_iter)
{
    GmArgs a;
    a.N = (long long)c->L * c->S;
    a.m = std::min(basis_size(c), max_iter);
    a.max_iter = max_iter;
    a.tol = c->cfg.gmres_tol;
    a.b = c->bhat; a.x = col.x; a.V = c->V; a.Z = c->Z; a.w = c->gw; a.h1 = c->h1; a.h2 = c->h2;
    a.red = c->red; a.partials = c->partials; a.counter = c->counter; a.gm = c->gm; a.ctl = ctl;
    a.skip_solve = skip;
    a.role = 2;
    a.reuse_max_iters = 0;
    const double *rowd = c->rowd;
    a.matvec = [col, ctl, rowd](const double *x, double *y, const int *sk, cudaStream_t s) {
        launch_jv(col, ctl, x, y, rowd, sk, s);
    };
    a.precond = [c, plan, ctl, rowd](const double *v, double *z, const int *sk, cudaStream_t s) {
        solve64(c, plan, v, z, ctl, s, rowd, sk, nullptr);
    };
    enqueue_fgmres(a, c->st);
}

// Enqueue thermochemistry, rates, photolysis, residual, Jacobian and the linear solve for state col.n (or n_override),
// writing the unscaled delta into delta_out.  ctl gates every kernel.
int enqueue_linear_step(xk_ctx *c, const double *n, double dt_override, double *delta_out, Ctl *ctl)
{
    Col col = c->col;
    col.n = const_cast<double *>(n);
    cudaStream_t st = c->st;
    // Gibbs energies and rate coefficients depend on the atmosphere only: evaluated once
    if (!c->rates_valid) {
        PhaseMark m(c, XK_PH_RATES);
        launch_rates(col, st);
        c->rates_valid = true;
    }
    { PhaseMark m(c, XK_PH_PHOTO); launch_photolysis(col, n, st); }
    { PhaseMark m(c, XK_PH_REACTION); launch_reaction_terms(col, n, st); }
    { PhaseMark m(c, XK_PH_RESIDUAL); launch_residual(col, n, col.F, ctl, c->cfg.f_floor, st); }
    cudaError_t e;
    const long long N = (long long)c->L * c->S;
    const int refine = std::max(c->cfg.refine_max_iter, 0);
    if (c->cfg.precision == XK_PREC_FP64) {
        {
            PhaseMark m(c, XK_PH_JACOBIAN);
            launch_jacobian64(col, n, ctl, dt_override, 1, c->A64, c->lo64, c->up64, st);
            if (refine > 0) {
                launch_diag(col, ctl, c->rowd, st);
                launch_rowdiv(N, col.b, c->rowd, c->bhat, st);
            }
        }
        { PhaseMark m(c, XK_PH_FACTOR); e = launch_factor<double>(sys64(c), c->plan, ctl, st); }
        if (e != cudaSuccess) return fail(c, XK_ECUDA, "factor launch: %s", cudaGetErrorString(e));
        PhaseMark m(c, XK_PH_SOLVE);
        if (refine > 0)
            enqueue_refine64(c, col, ctl, c->plan, nullptr, refine);
        else
            e = solve64(c, c->plan, col.b, col.x, ctl, st, nullptr, nullptr, nullptr);
        if (e != cudaSuccess) return fail(c, XK_ECUDA, "solve launch: %s", cudaGetErrorString(e));
    } else {
        if (dt_override > 0.0) return fail(c, XK_EINVAL, "mixed path reads dt from the control block");
        launch_route(ctl, st);
        const int *skip32 = &ctl->skip32;
        {
            PhaseMark m(c, XK_PH_JACOBIAN);
            launch_jacobian32(col, n, ctl, c->A32, c->lo32, c->up32, nullptr, st, skip32,
                              c->use_bcr ? (long long)c->bcr.Sp * c->bcr.Sp : 0);
            // equations divided by their diagonal: residuals in units of relative change per species
            launch_diag(col, ctl, c->rowd, st);
            launch_rowdiv(N, col.b, c->rowd, c->bhat, st);
        }
        {
            PhaseMark m(c, XK_PH_FACTOR);
            e = factor32(c, ctl, skip32);
        }
        if (e != cudaSuccess) return fail(c, XK_ECUDA, "factor launch: %s", cudaGetErrorString(e));
        GmArgs a;
        a.N = N;
        a.m = std::min(std::max(c->cfg.gmres_restart, 1), kMaxBasis);
        a.max_iter = std::max(c->cfg.gmres_max_iter, 1);
        a.tol = c->cfg.gmres_tol;
        a.b = c->bhat; a.x = col.x; a.V = c->V; a.Z = c->Z; a.w = c->gw; a.h1 = c->h1; a.h2 = c->h2;
        a.red = c->red; a.partials = c->partials; a.counter = c->counter; a.gm = c->gm; a.ctl = ctl;
        a.reuse_max_iters = c->cfg.reuse_max_iters > 0 ? c->cfg.reuse_max_iters : 40;
        FactorPlan plan64 = c->plan64;
        const double *rowd = c->rowd, *pin = c->pin, *pout = c->pout;
        a.matvec = [col, ctl, rowd](const double *x, double *y, const int *skip, cudaStream_t s) {
            launch_jv(col, ctl, x, y, rowd, skip, s);
        };
        // FGMRES around the FP32 inversion
        a.skip_solve = skip32;
        a.role = 0;
        a.precond = [c, ctl, rowd](const double *v, double *z, const int *skip, cudaStream_t s) {
            solve32(c, v, z, ctl, s, rowd, skip);
        };
        { PhaseMark m(c, XK_PH_SOLVE); enqueue_fgmres(a, st); }
        // FGMRES around the last FP64 factorization, rescaled to this step's variables
        if (c->cfg.reuse_factorization) {
            launch_reuse_scales(N, rowd, col.s, c->s64, c->pin, c->pout, ctl, st);
            a.skip_solve = &ctl->skip_reuse;
            a.role = 1;
            a.precond = [c, plan64, ctl, pin, pout](const double *v, double *z, const int *skip, cudaStream_t s) {
                solve64(c, plan64, v, z, ctl, s, pin, skip, pout);
            };
            { PhaseMark m(c, XK_PH_SOLVE); enqueue_fgmres(a, st); }
        }
        // FP64 factorization, then FGMRES refinement around it (or a direct solve), gated on the
        // device by ctl->skip64
        const int *skip64 = &ctl->skip64;
        {
            PhaseMark m(c, XK_PH_FALLBACK);
            launch_jacobian64(col, n, ctl, 0.0, 1, c->A64, c->lo64, c->up64, st, skip64);
            e = launch_factor<double>(sys64(c), c->plan64, ctl, st, skip64);
            if (e == cudaSuccess) {
                launch_after_refactor(N, col.s, c->s64, ctl, st);
                if (refine > 0)
                    enqueue_refine64(c, col, ctl, c->plan64, skip64, refine);
                else
                    e = solve64(c, c->plan64, col.b, col.x, ctl, st, nullptr, skip64, nullptr);
            }
        }
        if (e != cudaSuccess) return fail(c, XK_ECUDA, "FP64 fallback launch: %s", cudaGetErrorString(e));
    }
    launch_unscale(col, col.x, delta_out, st);
    return cuda_check(c, "step enqueue");
}

int enqueue_step(xk_ctx *c)
{
    Policy pol = policy_of(c->cfg);
    launch_begin(c->ctl, c->st);
    int rc = enqueue_linear_step(c, c->col.n, 0.0, c->col.delta, c->ctl);
    if (rc) return rc;
    {
        PhaseMark m(c, XK_PH_CONTROL);
        launch_check(c->col, c->ctl, pol, c->st);
        launch_decide(c->col, c->ctl, pol, c->st);
        launch_apply(c->col, c->ctl, c->st);
    }
    return cuda_check(c, "step enqueue");
}

int read_ctl(xk_ctx *c, Ctl *out)
{
    cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "sync: %s", cudaGetErrorString(e));
    *out = *c->ctl_host;
    return XK_OK;
}

// ---------------------------------------------------------------- CUDA graphs of steps

std::atomic<long long> g_graph_launches{0};

void drop_graphs(xk_ctx *c)
{
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

// Replay captured steps (tracing times each phase from the host instead).
bool graphs_on(const xk_ctx *c) { return c->cfg.use_graphs != 0 && !c->prof; }

// Rate coefficients depend on the atmosphere only: evaluated outside any graph, once.
void ensure_rates(xk_ctx *c)
{
    if (c->rates_valid) return;
    launch_rates(c->col, c->st);
    c->rates_valid = true;
}

// Enqueue `steps` controlled steps of c, and with ctl_copy the copy of its control block to the
// host mirror, into a graph being captured on the stream c->st.
int enqueue_chunk(xk_ctx *c, int steps, bool ctl_copy)
{
    for (int i = 0; i < steps; ++i) {
        int rc = enqueue_step(c);
        if (rc) return rc;
    }
    if (ctl_copy) cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    return XK_OK;
}

// End a capture begun on st and instantiate it; the kernels enqueued since n0 are nodes, not
// launches, until the graph is replayed.
int finish_capture(xk_ctx *c, cudaStream_t st, int rc, long long n0, cudaGraphExec_t *exec, long long *kernels)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    *kernels = launches() - n0;
    count_launches(-*kernels);
    *exec = nullptr;
    if (rc != XK_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != XK_OK ? rc : fail(c, XK_ECUDA, "step capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        cudaGetLastError();
        return fail(c, XK_ECUDA, "step graph instantiation: %s", cudaGetErrorString(e));
    }
    return XK_OK;
}

// The context's graph of `steps` steps (captured on first use), or null with *rc set.
StepGraph *step_graph(xk_ctx *c, int steps, bool ctl_copy, int *rc)
{
    *rc = XK_OK;
    for (auto &g : c->graphs)
        if (g.steps == steps && g.ctl_copy == ctl_copy) return &g;
    ensure_rates(c);
    if (!c->cap_st && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        *rc = cuda_check(c, "capture stream");
        return nullptr;
    }
    // captured on a stream of its own, replayed on the context's
    cudaStream_t own = c->st;
    c->st = c->cap_st;
    const long long n0 = launches();
    cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        c->st = own;
        *rc = fail(c, XK_ECUDA, "begin capture: %s", cudaGetErrorString(e));
        return nullptr;
    }
    int erc = enqueue_chunk(c, steps, ctl_copy);
    StepGraph g;
    g.steps = steps;
    g.ctl_copy = ctl_copy;
    *rc = finish_capture(c, c->st, erc, n0, &g.exec, &g.kernels);
    c->st = own;
    if (*rc) return nullptr;
    c->graphs.push_back(g);
    return &c->graphs.back();
}

int replay(xk_ctx *c, const StepGraph &g, cudaStream_t st)
{
    cudaError_t e = cudaGraphLaunch(g.exec, st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    count_launches(g.kernels);
    g_graph_launches.fetch_add(1, std::memory_order_relaxed);
    return XK_OK;
}

// `steps` controlled steps on c->st: one graph launch when graphs are on, else launched one by one.
int run_steps(xk_ctx *c, int steps, bool ctl_copy)
{
    if (!graphs_on(c)) {
        int rc = enqueue_chunk(c, steps, false);
        if (!rc && ctl_copy) cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
        return rc;
    }
    ensure_rates(c);
    int rc;
    StepGraph *g = step_graph(c, steps, ctl_copy, &rc);
    if (!g) return rc;
    return replay(c, *g, c->st);
}

}  // namespace

extern "C" {

int xk_version(void) { return 100; }

int xk_config_init(xk_config *cfg)
{
    if (!cfg) return XK_EINVAL;
    memset(cfg, 0, sizeof *cfg);
    cfg->precision = XK_PREC_FP64;
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->dt_max = 1e8; cfg->rel_reject = 1.0; cfg->rel_target = 0.5; cfg->grow_max = 3.0; cfg->shrink_min = 0.5;
    cfg->neg_tol = 1e-12; cfg->f_floor = 1e-20; cfg->dt_min = 1e-20; cfg->ss_dt = 1e8; cfg->ss_tol = 1e-3;
    cfg->gmres_restart = 30; cfg->gmres_max_iter = 40; cfg->gmres_tol = 1e-15;
    cfg->panel_width = 0; cfg->factor_ctas = 0; cfg->twisted = 1; cfg->reuse_max_iters = 40;
    cfg->refine_max_iter = 10;
    cfg->fp32_bcr = 1;
    cfg->wait_polls = 0;
    cfg->use_graphs = 1;
    cfg->photo_jacobian = 0;
    return XK_OK;
}

int xk_create(xk_ctx **out, const xk_config *cfg)
{
    if (!out) return XK_EINVAL;
    *out = nullptr;
    xk_config def;
    xk_config_init(&def);
    const xk_config &c = cfg ? *cfg : def;
    if (c.precision != XK_PREC_FP64 && c.precision != XK_PREC_MIXED) return XK_EINVAL;
    if (!(c.dt_max > 0) || !(c.dt_min > 0) || !(c.rel_reject > 0) || !(c.rel_target > 0)) return XK_EINVAL;
    if (c.gmres_restart > kMaxBasis) return XK_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    xk_ctx *x = new xk_ctx();
    x->cfg = c;
    x->st = (cudaStream_t)c.stream;
    cudaSetDevice(c.device);
    if (cudaMallocHost((void **)&x->ctl_host, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&x->parcel_host, sizeof(ParcelState)) != cudaSuccess) {
        cudaGetLastError();
        if (x->ctl_host) cudaFreeHost(x->ctl_host);
        delete x;
        return XK_ECUDA;
    }
    *out = x;
    return XK_OK;
}

int xk_destroy(xk_ctx *ctx)
{
    if (!ctx) return XK_EINVAL;
    drop_graphs(ctx);
    if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
    for (auto &v : ctx->ev)
        for (auto &pr : v) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
    if (ctx->parcel_host) cudaFreeHost(ctx->parcel_host);
    delete ctx;
    return XK_OK;
}

const char *xk_last_error(const xk_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int xk_load_network(xk_ctx *c, int S, int E, int R, const int *elem, const double *mass, const int *rtype,
                    const int *reac, const int *prod, const double *arr, const double *troe, const int *form,
                    const double *nasa)
{
    if (!c) return XK_EINVAL;
    if (S <= 0 || S > 65535 || E < 0 || R < 0 || R > (1 << 24)) return fail(c, XK_EINVAL, "bad sizes S=%d E=%d R=%d", S, E, R);
    if (!mass || !nasa || (R > 0 && (!rtype || !reac || !prod || !arr || !troe || !form)) || (E > 0 && !elem))
        return fail(c, XK_EINVAL, "null input array");
    for (int r = 0; r < R; ++r) {
        if (rtype[r] < 0 || rtype[r] > 2) return fail(c, XK_EINVAL, "reaction %d: bad type %d", r, rtype[r]);
        int nr = 0, np = 0;
        for (int s = 0; s < 3; ++s) {
            if (reac[3 * r + s] >= S || reac[3 * r + s] < -1 || prod[3 * r + s] >= S || prod[3 * r + s] < -1)
                return fail(c, XK_EINVAL, "reaction %d: species index out of range", r);
            nr += reac[3 * r + s] >= 0;
            np += prod[3 * r + s] >= 0;
        }
        if (nr == 0 || (rtype[r] != XK_RX_PHOTO && np == 0) || (rtype[r] == XK_RX_PHOTO && nr != 1))
            return fail(c, XK_EINVAL, "reaction %d: bad reactant/product count", r);
        for (int q = 0; q < 9; ++q)
            if (!std::isfinite(arr[9 * r + q])) return fail(c, XK_EINVAL, "reaction %d: non-finite rate parameter", r);
    }
    for (int y = 0; y < S; ++y)
        if (!(mass[y] > 0)) return fail(c, XK_EINVAL, "species %d: mass must be positive", y);
    c->S = S; c->E = E; c->R = R;
    c->elem.assign(elem, elem + (size_t)S * E);
    c->mass.assign(mass, mass + S);
    c->rtype.assign(rtype, rtype + R);
    c->reac.assign(reac, reac + 3 * (size_t)R);
    c->prod.assign(prod, prod + 3 * (size_t)R);
    c->arr.assign(arr, arr + 9 * (size_t)R);
    c->troe.assign(troe, troe + 4 * (size_t)R);
    c->form.assign(form, form + R);
    c->nasa.assign(nasa, nasa + 15 * (size_t)S);
    c->have_net = true;
    c->rates_valid = false;
    c->have_photo = false;
    c->ready = false;
    c->Rph = 0;
    c->prow.assign(R, -1);
    return XK_OK;
}

int xk_load_photo(xk_ctx *c, int W, int Rph, const int *prow, const double *lambda, const double *dlambda,
                  const double *J0, const double *sigma, const double *sigma_abs, double mu, double tf)
{
    if (!c) return XK_EINVAL;
    if (!c->have_net) return fail(c, XK_EINVAL, "load the network first");
    if (W < 0 || Rph < 0) return fail(c, XK_EINVAL, "bad sizes");
    if (!prow) return fail(c, XK_EINVAL, "null prow");
    if (W > 0 && (!lambda || !dlambda || !J0 || !sigma_abs || (Rph > 0 && !sigma))) return fail(c, XK_EINVAL, "null input array");
    if (!(mu > 0.0)) return fail(c, XK_EINVAL, "mu must be positive");
    int nph = 0;
    for (int r = 0; r < c->R; ++r) {
        if (c->rtype[r] == XK_RX_PHOTO) {
            if (prow[r] < 0 || prow[r] >= Rph) return fail(c, XK_EINVAL, "photolysis reaction %d: bad sigma row", r);
            ++nph;
        } else if (prow[r] != -1) {
            return fail(c, XK_EINVAL, "reaction %d is not photolysis but has a sigma row", r);
        }
    }
    if (W != c->W) c->sigma_s.clear();   // scattering cross sections belong to the old grid
    c->W = W; c->Rph = Rph;
    c->prow.assign(prow, prow + c->R);
    c->lam.assign(lambda, lambda + W);
    c->dlam.assign(dlambda, dlambda + W);
    c->J0.assign(J0, J0 + W);
    c->sigma.assign(sigma, sigma + (size_t)Rph * W);
    c->sigma_abs.assign(sigma_abs, sigma_abs + (size_t)c->S * W);
    c->mu = mu; c->tf = tf;
    c->have_photo = true;
    c->ready = false;
    (void)nph;
    return XK_OK;
}

int xk_load_scattering(xk_ctx *c, int W, const double *sigma_s, double albedo, int diffuse)
{
    if (!c) return XK_EINVAL;
    if (!c->have_photo) return fail(c, XK_EINVAL, "load the photolysis inputs first");
    if (W != c->W) return fail(c, XK_EINVAL, "scattering grid of %d bins, photolysis grid of %d", W, c->W);
    if (!(albedo >= 0.0 && albedo <= 1.0)) return fail(c, XK_EINVAL, "albedo must lie in [0, 1]");
    if (diffuse != 0 && diffuse != 1) return fail(c, XK_EINVAL, "diffuse must be 0 or 1");
    if (sigma_s) {
        for (size_t i = 0; i < (size_t)c->S * W; ++i)
            if (!(sigma_s[i] >= 0.0) || !std::isfinite(sigma_s[i]))
                return fail(c, XK_EINVAL, "scattering cross sections must be finite and non-negative");
        c->sigma_s.assign(sigma_s, sigma_s + (size_t)c->S * W);
    } else {
        c->sigma_s.clear();
    }
    c->albedo = albedo;
    c->diffuse = diffuse;
    c->ready = false;
    return XK_OK;
}

int xk_load_atmosphere(xk_ctx *c, int L, const double *P_bar, const double *T, const double *Kzz,
                       const double *dcoef, double g, double mbar, double alpha_T)
{
    if (!c) return XK_EINVAL;
    if (!c->have_net) return fail(c, XK_EINVAL, "load the network first");
    if (L <= 0) return fail(c, XK_EINVAL, "L must be positive");
    if (!P_bar || !T || !Kzz || !dcoef) return fail(c, XK_EINVAL, "null input array");
    for (int k = 0; k < L; ++k) {
        if (!(P_bar[k] > 0) || !(T[k] > 0) || !(Kzz[k] >= 0)) return fail(c, XK_EINVAL, "layer %d: bad P/T/Kzz", k);
        if (k > 0 && !(P_bar[k] < P_bar[k - 1])) return fail(c, XK_EINVAL, "pressure must fall with layer index");
    }
    if (!(g > 0) || !(mbar > 0)) return fail(c, XK_EINVAL, "g and mbar must be positive");
    c->L = L;
    c->P.assign(P_bar, P_bar + L);
    c->T.assign(T, T + L);
    c->Kzz.assign(Kzz, Kzz + L);
    c->dcoef.assign(dcoef, dcoef + c->S);
    c->g = g; c->mbar = mbar; c->alpha_T = alpha_T;
    c->have_atm = true;
    c->rates_valid = false;
    c->ready = false;
    return XK_OK;
}

int xk_workspace_bytes(xk_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return XK_EINVAL;
    if (!c->have_net || !c->have_atm) return fail(c, XK_EINVAL, "load network and atmosphere first");
    bool has_photo = false;
    for (int r = 0; r < c->R; ++r) has_photo |= c->rtype[r] == XK_RX_PHOTO;
    if (has_photo && !c->have_photo) return fail(c, XK_EINVAL, "network has photolysis reactions: load photolysis inputs");
    build_indices(c);
    *bytes = layout(c, nullptr);
    return XK_OK;
}

int xk_set_workspace(xk_ctx *c, void *dptr, size_t bytes)
{
    size_t need = 0;
    int rc = xk_workspace_bytes(c, &need);
    if (rc) return rc;
    if (!dptr || bytes < need) return fail(c, XK_ENOMEM, "workspace of %zu bytes, need %zu", bytes, need);
    if (((uintptr_t)dptr) & 255) return fail(c, XK_EINVAL, "workspace must be 256-byte aligned");
    if (c->cfg.photo_jacobian && c->diffuse)
        return fail(c, XK_EINVAL, "photo_jacobian differentiates the direct beam only: not with the diffuse field");
    cudaSetDevice(c->cfg.device);
    drop_graphs(c);
    c->ws = (char *)dptr;
    c->ws_bytes = bytes;
    layout(c, c->ws);
    int sz = c->cfg.precision == XK_PREC_FP64 ? 8 : 4;
    int nbh = c->cfg.panel_width;
    if (sz == 4 && !c->cfg.fp32_pivoting && nbh != 16) nbh = 32;   // grid kernel widths (8 is cluster-only)
    if (sz == 8 && nbh == 0) nbh = 8;
    if (factor_plan(c->S, sz, nbh, c->cfg.factor_ctas, &c->plan) != 0)
        return fail(c, XK_EINVAL, "no factorization plan for S=%d (panel %d)", c->S, c->cfg.panel_width);
    // FP64 factorization (the path itself, or the fallback of the mixed path): the context's
    // panel width and CTA count in FP64 mode
    const int nb64 = sz == 8 ? nbh : 8;
    if (factor_plan(c->S, 8, nb64, sz == 8 ? c->cfg.factor_ctas : 0, &c->plan64) != 0)
        return fail(c, XK_EINVAL, "no FP64 factorization plan for S=%d", c->S);
    c->use_cluster = false;
    c->use_cluster_solve = false;
    c->use_bcr = sz == 4 && c->cfg.fp32_bcr;
    c->use_cluster_solve64 = c->cfg.cluster_size >= 0 && solve_cluster_plan(c->S, 8, &c->splan64) == 0;
    set_preview(c, &c->plan64);
    if (sz == 8) set_preview(c, &c->plan);
    if (c->use_bcr) {
        if (bcr_build(c->bcr, c->L, c->S, c->st) != 0)
            return fail(c, XK_ECUDA, "block cyclic reduction plan: %s", cudaGetErrorString(cudaGetLastError()));
        // padded blocks: zero, then the identity in the padding rows (callers may fill only S x S)
        cudaMemsetAsync(c->A32, 0, sizeof(float) * (size_t)c->L * c->bcr.Sp * c->bcr.Sp, c->st);
        bcr_init_pad(c->bcr, c->st);
    } else if (sz == 4 && !c->cfg.fp32_pivoting && c->cfg.cluster_size >= 0) {
        const int nbc = c->cfg.panel_width == 16 ? 16 : 8;
        // the panel rows go through gbuf (4 x S x 32 floats, enough for 4 x 16 x round_up(S, 4))
        if (cluster_plan(c->S, nbc, c->cfg.cluster_size, &c->cplan) == 0 &&
            cluster_ubuf_floats(c->cplan) <= 4 * (size_t)c->S * 32) {
            c->use_cluster = true;
            c->use_cluster_solve = solve_cluster_plan(c->S, 4, &c->splan) == 0;
            // inverses from both ends need the matching sweeps
            if (!(c->use_cluster_solve && c->splan.twisted) || c->cfg.twisted == 0) c->cplan.twisted = 0;
        }
        else if (c->cfg.cluster_size > 0)
            return fail(c, XK_EINVAL, "no cluster of %d CTAs holds the S=%d block (panel %d)", c->cfg.cluster_size,
                        c->S, nbc);
    }
    Col &k = c->col;
    up(c, k.elem, c->elem);
    up(c, c->pgraph.gp, c->pg_p); up(c, c->pgraph.gv, c->pg_v); up(c, c->pgraph.gs, c->pg_s);
    up(c, c->pgraph.gcode, c->pg_code);
    up(c, c->eqix.sp, c->eq_sp); up(c, c->eqix.se, c->eq_se); up(c, c->eqix.sc, c->eq_sc);
    up(c, c->eqix.ep, c->eq_ep); up(c, c->eqix.ey, c->eq_ey); up(c, c->eqix.ec, c->eq_ec);
    up(c, c->eqix.eij, c->eq_eij);
    up(c, k.mass, c->mass); up(c, k.nasa, c->nasa); up(c, k.dcoef, c->dcoef);
    up(c, k.arr, c->arr); up(c, k.troe, c->troe); up(c, k.rtype, c->rtype); up(c, k.reac, c->reac);
    up(c, k.prod, c->prod); up(c, k.form, c->form); up(c, k.prow, c->prow);
    up(c, k.yp, c->yp); up(c, k.yent, c->yent); up(c, k.jp, c->jp); up(c, k.jcol, c->jcol); up(c, k.jtp, c->jtp); up(c, k.jrs, c->jrs);
    up(c, k.jdq, c->jdq);
    up(c, k.J0, c->J0); up(c, k.dlam, c->dlam); up(c, k.sigma, c->sigma); up(c, k.sig_abs, c->sig_abs_c);
    up(c, k.abs_sp, c->abs_sp);
    up(c, k.sig_sca, c->sig_sca_c); up(c, k.sca_sp, c->sca_sp);
    up(c, k.P, c->P); up(c, k.T, c->T); up(c, k.Kzz, c->Kzz);
    cudaMemsetAsync(c->bar, 0, 8 * sizeof(unsigned), c->st);
    if (c->counter) cudaMemsetAsync(c->counter, 0, 8 * sizeof(unsigned), c->st);
    cudaMemsetAsync(c->col.n, 0, sizeof(double) * (size_t)c->L * c->S, c->st);
    Ctl init = fresh_ctl(c);
    init.dt = 1e-8;
    init.dt_fp64 = 1e300;
    init.reuse_enabled = c->cfg.reuse_factorization;
    *c->ctl_host = init;
    cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->ctl_aux, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    launch_grid(c->col, c->st);
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "upload: %s", cudaGetErrorString(e));
    c->ready = true;
    c->rates_valid = false;
    return cuda_check(c, "set_workspace");
}

int xk_set_state(xk_ctx *c, const double *n, int on_device)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n) return fail(c, XK_EINVAL, "null state");
    cudaMemcpyAsync(c->col.n, n, sizeof(double) * (size_t)c->L * c->S,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "set_state");
    return cuda_check(c, "set_state");
}

int xk_set_mixing_ratios(xk_ctx *c, const double *f, int on_device)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!f) return fail(c, XK_EINVAL, "null mixing ratios");
    cudaMemcpyAsync(c->col.tmp, f, sizeof(double) * (size_t)c->L * c->S,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st);
    launch_set_mixing(c->col, c->col.tmp, c->col.n, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "set_mixing_ratios");
    return cuda_check(c, "set_mixing_ratios");
}

int xk_get_state(xk_ctx *c, double *n, int on_device)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n) return fail(c, XK_EINVAL, "null output");
    cudaMemcpyAsync(n, c->col.n, sizeof(double) * (size_t)c->L * c->S,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "get_state");
    return cuda_check(c, "get_state");
}

static void fill_step_info(const Ctl &h, xk_step_info *info)
{
    if (!info) return;
    info->accepted = h.accepted;
    info->dt_used = h.last_dt;
    info->dt_next = h.dt;
    info->max_rel = h.max_rel;
    info->n_neg = h.n_neg;
    info->converged = h.converged;
    info->solver_iters = h.solver_iters;
    info->solver_resid = h.solver_resid;
    info->used_fp64 = h.used_fp64;
}

int xk_step(xk_ctx *c, double dt, xk_step_info *info)
{
    int rc = need_ready(c);
    if (rc) return rc;
    Ctl h;
    if ((rc = read_ctl(c, &h))) return rc;
    h.finished = 0;
    h.converged = 0;
    h.status = 0;
    h.err_timeout = 0;
    h.err_singular = 0;
    h.wait_polls = fresh_ctl(c).wait_polls;
    if (dt > 0.0) h.dt = dt;
    *c->ctl_host = h;
    cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    if ((rc = run_steps(c, 1, false))) return rc;
    if ((rc = read_ctl(c, &h))) return rc;
    fill_step_info(h, info);
    if (h.err_timeout) return timed_out(c);
    if (h.status) return fail(c, h.status, "step failed with status %d", h.status);
    return XK_OK;
}

int xk_run_to_steady(xk_ctx *c, double dt0, int max_steps, xk_run_info *info)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (max_steps <= 0) return fail(c, XK_EINVAL, "max_steps must be positive");
    Ctl h;
    if ((rc = read_ctl(c, &h))) return rc;
    Ctl init = fresh_ctl(c);
    init.dt = dt0 > 0.0 ? dt0 : h.dt;
    init.t = 0.0;
    init.dt_fp64 = h.dt_fp64;
    init.reuse_enabled = c->cfg.reuse_factorization;
    init.have64 = h.have64;
    *c->ctl_host = init;
    cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    int enq = 0;
    const int chunk = 16;
    while (enq < max_steps) {
        int nrun = std::min(chunk, max_steps - enq);
        if ((rc = run_steps(c, nrun, false))) return rc;
        enq += nrun;
        if ((rc = read_ctl(c, &h))) return rc;
        if (h.finished) break;
    }
    if (info) {
        info->converged = h.converged;
        info->steps = h.steps;
        info->accepted = h.n_acc;
        info->rejected = h.n_rej;
        info->t = h.t;
        info->dt = h.dt;
        info->max_rel = h.max_rel;
        info->solver_iters = h.total_iters;
        info->fp64_steps = h.fp64_steps;
        info->refactors = h.refactors;
    }
    if (h.err_timeout) return timed_out(c);
    if (h.status) return fail(c, h.status, "run stopped with status %d", h.status);
    if (!h.converged) return fail(c, XK_ENOCONV, "no steady state after %d steps", h.steps);
    return XK_OK;
}

// ---------------------------------------------------------------- rows

static int finish_eval(xk_ctx *c, const char *what)
{
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return cuda_check(c, what);
}

static void d2d(xk_ctx *c, void *dst, const void *src, size_t bytes)
{
    if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->st);
}

int xk_eval_grid(xk_ctx *c, double *ngas, double *z, double *dz, double *dzi)
{
    int rc = need_ready(c);
    if (rc) return rc;
    const size_t L = c->L;
    if (ngas) d2d(c, ngas, c->col.ngas, L * 8);
    if (z) d2d(c, z, c->col.z, L * 8);
    if (dz) d2d(c, dz, c->col.dz, L * 8);
    if (dzi && L > 1) d2d(c, dzi, c->col.dzi, (L - 1) * 8);
    return finish_eval(c, "eval_grid");
}

int xk_eval_thermo(xk_ctx *c, double *grt, double *lnkc)
{
    int rc = need_ready(c);
    if (rc) return rc;
    launch_rates(c->col, c->st);
    if (grt) d2d(c, grt, c->col.grt, (size_t)c->L * c->S * 8);
    if (lnkc) d2d(c, lnkc, c->col.lnkc, (size_t)c->L * c->R * 8);
    return finish_eval(c, "eval_thermo");
}

int xk_set_rate_coefficients(xk_ctx *c)
{
    int rc = need_ready(c);
    if (rc) return rc;
    launch_rates(c->col, c->st);
    c->rates_valid = true;
    return finish_eval(c, "set_rate_coefficients");
}

int xk_eval_rates(xk_ctx *c, double *kf, double *kr)
{
    int rc = need_ready(c);
    if (rc) return rc;
    launch_rates(c->col, c->st);
    if (kf) d2d(c, kf, c->col.kf, (size_t)c->L * c->R * 8);
    if (kr) d2d(c, kr, c->col.kr, (size_t)c->L * c->R * 8);
    return finish_eval(c, "eval_rates");
}

int xk_eval_photolysis(xk_ctx *c, const double *n, double *kph)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n || !kph) return fail(c, XK_EINVAL, "null pointer");
    launch_photolysis(c->col, n, c->st);
    d2d(c, kph, c->col.kph, (size_t)c->L * c->Rph * 8);
    return finish_eval(c, "eval_photolysis");
}

int xk_eval_transport(xk_ctx *c, double *u, double *v)
{
    int rc = need_ready(c);
    if (rc) return rc;
    size_t bytes = (size_t)(c->L - 1) * c->S * 8;
    if (u) d2d(c, u, c->col.u, bytes);
    if (v) d2d(c, v, c->col.v, bytes);
    return finish_eval(c, "eval_transport");
}

int xk_eval_residual(xk_ctx *c, const double *n, double *F)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n || !F) return fail(c, XK_EINVAL, "null pointer");
    launch_rates(c->col, c->st);
    launch_photolysis(c->col, n, c->st);
    launch_reaction_terms(c->col, n, c->st);
    launch_residual(c->col, n, F, nullptr, c->cfg.f_floor, c->st);
    return finish_eval(c, "eval_residual");
}

int xk_eval_jacobian(xk_ctx *c, const double *n, double dt, double *A, double *lo, double *up)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n || !A || !lo || !up || !(dt > 0)) return fail(c, XK_EINVAL, "bad argument");
    Col col = c->col;
    col.ld = c->S;
    launch_rates(col, c->st);
    launch_photolysis(col, n, c->st);
    launch_reaction_terms(col, n, c->st);
    launch_residual(col, n, col.F, nullptr, c->cfg.f_floor, c->st);
    launch_jacobian64(col, n, nullptr, dt, 0, A, lo, up, c->st);
    return finish_eval(c, "eval_jacobian");
}

int xk_block_solve(xk_ctx *c, const double *A, const double *lo, const double *up, const double *f, double *x)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!A || !lo || !up || !f || !x) return fail(c, XK_EINVAL, "null pointer");
    const size_t S = c->S, L = c->L;
    cudaMemcpy2DAsync(c->A64, c->col.ld * 8, A, S * 8, S * 8, L * S, cudaMemcpyDeviceToDevice, c->st);
    d2d(c, c->lo64, lo, L * S * 8);
    d2d(c, c->up64, up, L * S * 8);
    Ctl init = fresh_ctl(c);
    *c->ctl_host = init;
    cudaMemcpyAsync(c->ctl_aux, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    cudaError_t e = launch_factor<double>(sys64(c), c->plan64, c->ctl_aux, c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "factor launch: %s", cudaGetErrorString(e));
    e = solve64(c, c->plan64, f, x, c->ctl_aux, c->st, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "solve launch: %s", cudaGetErrorString(e));
    cudaMemcpyAsync(c->ctl_host, c->ctl_aux, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    if ((rc = finish_eval(c, "block_solve"))) return rc;
    if (c->ctl_host->err_timeout) return timed_out(c);
    if (c->ctl_host->err_singular) return fail(c, XK_ESINGULAR, "zero pivot in a diagonal block");
    return XK_OK;
}

int xk_block_solve32(xk_ctx *c, const double *A, const double *lo, const double *up, const double *f, double *x)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (c->cfg.precision != XK_PREC_MIXED) return fail(c, XK_EINVAL, "xk_block_solve32 needs a mixed-precision context");
    if (!A || !lo || !up || !f || !x) return fail(c, XK_EINVAL, "null pointer");
    const size_t S = c->S, L = c->L, ld = c->col.ld;
    if (c->use_bcr) {
        const size_t Sp = c->bcr.Sp;
        for (size_t k = 0; k < L; ++k) launch_convert32(A + k * S * S, S, c->A32 + k * Sp * Sp, Sp, S, S, c->st);
    } else {
        launch_convert32(A, S, c->A32, ld, L * S, S, c->st);
    }
    launch_convert32(lo, L * S, c->lo32, L * S, 1, L * S, c->st);
    launch_convert32(up, L * S, c->up32, L * S, 1, L * S, c->st);
    Ctl init = fresh_ctl(c);
    *c->ctl_host = init;
    cudaMemcpyAsync(c->ctl_aux, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    cudaError_t e = factor32(c, c->ctl_aux, nullptr);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "factor launch: %s", cudaGetErrorString(e));
    e = solve32(c, f, x, c->ctl_aux, c->st, nullptr, nullptr);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "solve launch: %s", cudaGetErrorString(e));
    cudaMemcpyAsync(c->ctl_host, c->ctl_aux, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    if ((rc = finish_eval(c, "block_solve32"))) return rc;
    if (c->ctl_host->err_timeout) return timed_out(c);
    if (c->ctl_host->err_singular) return fail(c, XK_ESINGULAR, "zero pivot in a diagonal block");
    return XK_OK;
}

int xk_step_delta(xk_ctx *c, const double *n, double dt, double *delta, int *iters, double *resid)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n || !delta || !(dt > 0)) return fail(c, XK_EINVAL, "bad argument");
    Ctl init = fresh_ctl(c);
    init.dt = dt;
    init.dt_fp64 = 1e300;
    *c->ctl_host = init;
    cudaMemcpyAsync(c->ctl_aux, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    double dto = c->cfg.precision == XK_PREC_FP64 ? dt : 0.0;
    if ((rc = enqueue_linear_step(c, n, dto, delta, c->ctl_aux))) return rc;
    cudaMemcpyAsync(c->ctl_host, c->ctl_aux, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    if ((rc = finish_eval(c, "step_delta"))) return rc;
    if (iters) *iters = c->ctl_host->used_fp64 ? -1 : c->ctl_host->solver_iters;
    if (resid) *resid = c->ctl_host->solver_resid;
    if (c->ctl_host->err_timeout) return timed_out(c);
    if (c->ctl_host->err_singular) return fail(c, XK_ESINGULAR, "zero pivot in a diagonal block");
    return XK_OK;
}

int xk_hold_next_barrier(xk_ctx *c)
{
    int rc = need_ready(c);
    if (rc) return rc;
    // arrival counts that a grid of at most 2^30 CTAs never completes, for both counter pairs
    // (the whole grid, and the second half of a two-chain elimination)
    const unsigned held[4] = {1u << 30, 0u, 1u << 30, 0u};
    cudaMemcpyAsync(c->bar, held, sizeof held, cudaMemcpyHostToDevice, c->st);
    return finish_eval(c, "hold_next_barrier");
}

int xk_factor_work(xk_ctx *c, double *mma_flops, double *leaf_flops)
{
    if (!c || !c->ready || !c->use_bcr) return XK_EINVAL;
    bcr_work(c->bcr, mma_flops, leaf_flops);
    return XK_OK;
}

long long xk_launch_count(void) { return launches(); }

long long xk_graph_launch_count(void) { return g_graph_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------- batches

struct BatchSlot {
    xk_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;      // end of the steps submitted last (xk_batch_submit)
    bool inflight = false;
    cudaStream_t saved_st = nullptr;
    FactorPlan saved_plan{}, saved_plan64{};
    int saved_solve_ctas = 0;
    size_t bytes = 0;
    bool finished = false;
};

}  // extern "C"

struct xk_batch {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 1;
    std::vector<BatchSlot> slots;
    std::string err;
    // one round of xk_batch_step for every unfinished column, captured as one graph: a branch per
    // column from a fork on `origin`, joined back there
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t round = nullptr;
    std::vector<int> round_slots;
    int round_steps = 0;
    long long round_kernels = 0;
};

namespace {

void drop_round(xk_batch *b)
{
    if (b->round) cudaGraphExecDestroy(b->round);
    b->round = nullptr;
    b->round_slots.clear();
    b->round_steps = 0;
    b->round_kernels = 0;
}

// Capture nsteps steps of every listed slot's column, each on its slot's stream, into b->round.
int capture_round(xk_batch *b, const std::vector<int> &live, int nsteps)
{
    drop_round(b);
    cudaError_t e = cudaSuccess;
    if (!b->origin) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    while (e == cudaSuccess && b->joins.size() < b->slots.size()) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->joins.push_back(ev);
    }
    if (e != cudaSuccess) {
        b->err = std::string("batch graph: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return XK_ECUDA;
    }
    for (int i : live) ensure_rates(b->slots[i].ctx);
    const long long n0 = launches();
    e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        b->err = std::string("batch capture: ") + cudaGetErrorString(e);
        return XK_ECUDA;
    }
    cudaEventRecord(b->fork, b->origin);
    int rc = XK_OK;
    xk_ctx *bad = nullptr;
    for (int i : live) {
        BatchSlot &s = b->slots[i];
        cudaStreamWaitEvent(s.st, b->fork, 0);
        if (rc == XK_OK && (rc = enqueue_chunk(s.ctx, nsteps, true)) != XK_OK) bad = s.ctx;
        cudaEventRecord(b->joins[i], s.st);
        cudaStreamWaitEvent(b->origin, b->joins[i], 0);
    }
    xk_ctx *owner = bad ? bad : b->slots[live[0]].ctx;
    rc = finish_capture(owner, b->origin, rc, n0, &b->round, &b->round_kernels);
    if (rc) {
        b->err = owner->err;
        drop_round(b);
        return rc;
    }
    b->round_slots = live;
    b->round_steps = nsteps;
    return XK_OK;
}

}  // namespace

extern "C" {

int xk_batch_create(xk_batch **out, int device, size_t budget_bytes, int max_slots)
{
    if (!out || max_slots <= 0 || budget_bytes == 0) return XK_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return XK_ECUDA;
    }
    xk_batch *b = new xk_batch();
    b->device = device;
    b->budget = budget_bytes;
    b->max_slots = max_slots;
    b->slots.resize(max_slots);
    *out = b;
    return XK_OK;
}

int xk_batch_remove(xk_batch *b, int slot)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].ctx) return XK_EINVAL;
    BatchSlot &s = b->slots[slot];
    cudaSetDevice(b->device);
    cudaStreamSynchronize(s.st);
    drop_graphs(s.ctx);
    drop_round(b);
    s.ctx->st = s.saved_st;
    s.ctx->plan = s.saved_plan;
    s.ctx->plan64 = s.saved_plan64;
    s.ctx->bcr.solve_ctas = s.saved_solve_ctas;
    if (s.ev) cudaEventDestroy(s.ev);
    cudaStreamDestroy(s.st);
    b->used -= s.bytes;
    s = BatchSlot();
    return cuda_check(nullptr, "batch_remove");
}

int xk_batch_destroy(xk_batch *b)
{
    if (!b) return XK_EINVAL;
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (b->slots[i].ctx) xk_batch_remove(b, i);
    drop_round(b);
    for (auto ev : b->joins) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
    return XK_OK;
}

int xk_batch_add(xk_batch *b, xk_ctx *c, double dt0, int *slot)
{
    if (!b || !c || !slot || !(dt0 > 0)) return XK_EINVAL;
    int rc = need_ready(c);
    if (rc) return rc;
    if (c->cfg.device != b->device) return fail(c, XK_EINVAL, "context and batch are on different devices");
    for (auto &s : b->slots)
        if (s.ctx == c) return fail(c, XK_EINVAL, "context is already in this batch");
    int free_slot = -1;
    for (int i = 0; i < (int)b->slots.size() && free_slot < 0; ++i)
        if (!b->slots[i].ctx) free_slot = i;
    if (free_slot < 0) return fail(c, XK_ENOMEM, "all %d batch slots are taken", b->max_slots);
    if (b->used + c->ws_bytes > b->budget)
        return fail(c, XK_ENOMEM, "footprint %zu bytes does not fit the remaining budget %zu", c->ws_bytes,
                    b->budget - b->used);
    cudaSetDevice(b->device);
    BatchSlot &s = b->slots[free_slot];
    if (cudaStreamSynchronize(c->st) != cudaSuccess || cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_check(c, "batch_add");
    if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(s.st);
        s = BatchSlot();
        return cuda_check(c, "batch_add");
    }
    // a share of the SMs for this column's persistent kernels
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    int share = std::max(1, sms / b->max_slots);
    FactorPlan p, p64;
    int sz = c->cfg.precision == XK_PREC_FP64 ? 8 : 4;
    if (factor_plan(c->S, sz, c->plan.nb, share, &p) != 0 || factor_plan(c->S, 8, c->plan64.nb, share, &p64) != 0) {
        cudaEventDestroy(s.ev);
        cudaStreamDestroy(s.st);
        s = BatchSlot();
        return fail(c, XK_EINVAL, "no factorization plan for a %d-CTA share", share);
    }
    set_preview(c, &p64);
    if (sz == 8) set_preview(c, &p);
    drop_graphs(c);
    drop_round(b);
    s.ctx = c;
    s.saved_st = c->st;
    s.saved_plan = c->plan;
    s.saved_plan64 = c->plan64;
    s.saved_solve_ctas = c->bcr.solve_ctas;
    c->bcr.solve_ctas = share;          // the reduction's cooperative solve on this column's share of the SMs
    s.bytes = c->ws_bytes;
    s.finished = false;
    c->st = s.st;
    c->plan = p;
    c->plan64 = p64;
    b->used += s.bytes;
    Ctl h;
    if ((rc = read_ctl(c, &h))) return rc;
    Ctl init = fresh_ctl(c);
    init.dt = dt0;
    init.dt_fp64 = 1e300;
    init.reuse_enabled = c->cfg.reuse_factorization;
    *c->ctl_host = init;
    cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    *slot = free_slot;
    return cuda_check(c, "batch_add");
}

int xk_batch_step(xk_batch *b, int nsteps)
{
    if (!b || nsteps <= 0) return XK_EINVAL;
    cudaSetDevice(b->device);
    // round-robin so that every column's next step is queued before the following ones
    b->err.clear();
    for (auto &s : b->slots)
        if (s.ctx && s.inflight) {
            b->err = "a slot has submitted steps in flight (query it first)";
            return XK_EINVAL;
        }
    std::vector<int> live;
    bool graphs = true;
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (b->slots[i].ctx && !b->slots[i].finished) {
            live.push_back(i);
            graphs = graphs && graphs_on(b->slots[i].ctx);
        }
    if (live.empty()) return XK_OK;
    if (graphs) {
        // one graph launch for the whole round, captured again when the set of columns changes
        if (!b->round || b->round_slots != live || b->round_steps != nsteps) {
            int rc = capture_round(b, live, nsteps);
            if (rc) return rc;
        }
        for (int i : live) ensure_rates(b->slots[i].ctx);
        cudaError_t e = cudaGraphLaunch(b->round, b->origin);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
        if (e != cudaSuccess) {
            b->err = std::string("batch round: ") + cudaGetErrorString(e);
            return XK_ECUDA;
        }
        count_launches(b->round_kernels);
        g_graph_launches.fetch_add(1, std::memory_order_relaxed);
        for (int i : live) b->slots[i].finished = b->slots[i].ctx->ctl_host->finished != 0;
        return cuda_check(nullptr, "batch_step");
    }
    for (int k = 0; k < nsteps; ++k)
        for (int i : live) {
            BatchSlot &s = b->slots[i];
            int rc = enqueue_step(s.ctx);
            if (rc) {
                b->err = s.ctx->err;
                return rc;
            }
        }
    for (int i : live) {
        BatchSlot &s = b->slots[i];
        cudaMemcpyAsync(s.ctx->ctl_host, s.ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s.st);
    }
    for (int i : live) {
        BatchSlot &s = b->slots[i];
        cudaError_t e = cudaStreamSynchronize(s.st);
        if (e != cudaSuccess) {
            int rc = fail(s.ctx, XK_ECUDA, "batch step: %s", cudaGetErrorString(e));
            b->err = s.ctx->err;
            return rc;
        }
        s.finished = s.ctx->ctl_host->finished != 0;
    }
    return cuda_check(nullptr, "batch_step");
}

const char *xk_batch_last_error(xk_batch *b) { return b ? b->err.c_str() : "null batch"; }

int xk_batch_fits(xk_batch *b, size_t bytes, int *fits)
{
    if (!b || !fits) return XK_EINVAL;
    bool slot = false;
    for (const auto &s : b->slots) slot |= s.ctx == nullptr;
    *fits = (slot && b->used + bytes <= b->budget) ? 1 : 0;
    return XK_OK;
}

int xk_batch_submit(xk_batch *b, int slot, int nsteps)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].ctx || nsteps <= 0) return XK_EINVAL;
    BatchSlot &s = b->slots[slot];
    if (s.inflight) {
        b->err = "steps already submitted to this slot";
        return XK_EINVAL;
    }
    if (s.finished) return XK_OK;
    cudaSetDevice(b->device);
    b->err.clear();
    int rc = run_steps(s.ctx, nsteps, true);
    if (rc) {
        b->err = s.ctx->err;
        return rc;
    }
    if (cudaEventRecord(s.ev, s.st) != cudaSuccess) {
        rc = fail(s.ctx, XK_ECUDA, "batch submit: %s", cudaGetErrorString(cudaGetLastError()));
        b->err = s.ctx->err;
        return rc;
    }
    s.inflight = true;
    return XK_OK;
}

int xk_batch_query(xk_batch *b, int slot, int *done)
{
    if (!b || !done || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].ctx) return XK_EINVAL;
    BatchSlot &s = b->slots[slot];
    *done = 1;
    if (!s.inflight) return XK_OK;
    cudaError_t e = cudaEventQuery(s.ev);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        *done = 0;
        return XK_OK;
    }
    s.inflight = false;
    if (e != cudaSuccess) {
        int rc = fail(s.ctx, XK_ECUDA, "batch query: %s", cudaGetErrorString(e));
        b->err = s.ctx->err;
        return rc;
    }
    s.finished = s.ctx->ctl_host->finished != 0;
    return XK_OK;
}

int xk_batch_poll(xk_batch *b, int slot, xk_run_info *info, int *finished, int *status)
{
    if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].ctx) return XK_EINVAL;
    const Ctl &h = *b->slots[slot].ctx->ctl_host;
    if (info) {
        info->converged = h.converged;
        info->steps = h.steps;
        info->accepted = h.n_acc;
        info->rejected = h.n_rej;
        info->t = h.t;
        info->dt = h.dt;
        info->max_rel = h.max_rel;
        info->solver_iters = h.total_iters;
        info->fp64_steps = h.fp64_steps;
        info->refactors = h.refactors;
    }
    if (finished) *finished = b->slots[slot].finished ? 1 : 0;
    if (status) *status = h.err_timeout ? XK_ETIMEOUT : h.status;
    return XK_OK;
}

// ------------------------------------------- equilibrium initial state and pathway analyser

int xk_equilibrium(xk_ctx *c, const double *b, double *x, int set_state, int max_iter, double tol,
                   xk_equilibrium_info *info)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (max_iter <= 0 || !(tol > 0.0)) return fail(c, XK_EINVAL, "equilibrium: bad max_iter or tol");
    if (c->E + 1 > 31) return fail(c, XK_EINVAL, "equilibrium: at most 30 elements");
    ensure_rates(c);   // G/RT of the atmosphere
    cudaError_t e = launch_equilibrium(c->col, c->eqix, b, x, set_state ? c->col.n : nullptr, max_iter, tol,
                                       c->eq_iters, c->eq_status, c->st);
    if (e != cudaSuccess) return fail(c, XK_EINVAL, "equilibrium launch: %s", cudaGetErrorString(e));
    std::vector<int> its(c->L), sts(c->L);
    cudaMemcpyAsync(its.data(), c->eq_iters, sizeof(int) * c->L, cudaMemcpyDeviceToHost, c->st);
    cudaMemcpyAsync(sts.data(), c->eq_status, sizeof(int) * c->L, cudaMemcpyDeviceToHost, c->st);
    rc = finish_eval(c, "equilibrium");
    if (rc) return rc;
    int worst = 0, bad = 0, sing = 0;
    for (int k = 0; k < c->L; ++k) {
        worst = std::max(worst, its[k]);
        bad += sts[k] == 1;
        sing += sts[k] < 0;
    }
    if (info) {
        info->iters_max = worst;
        info->layers_not_converged = bad;
        info->layers_singular = sing;
    }
    if (sing) return fail(c, XK_ESINGULAR, "equilibrium: %d layers with a singular system or no species", sing);
    if (bad) return fail(c, XK_ENOCONV, "equilibrium: %d layers not converged in %d iterations", bad, max_iter);
    return XK_OK;
}

int xk_reaction_fluxes(xk_ctx *c, const double *n, double *q)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!n || !q) return fail(c, XK_EINVAL, "null pointer");
    ensure_rates(c);
    launch_photolysis(c->col, n, c->st);
    launch_fluxes(c->col, n, q, c->st);
    return finish_eval(c, "reaction_fluxes");
}

int xk_pathways(xk_ctx *c, const double *q, int nsrc, const int *src, double *dist, int *pred_sp, int *pred_edge,
                int *lim_edge, double *lim_w)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!q || !src || nsrc <= 0 || nsrc > c->S) return fail(c, XK_EINVAL, "pathways: bad sources");
    if ((lim_edge == nullptr) != (lim_w == nullptr))
        return fail(c, XK_EINVAL, "pathways: lim_edge and lim_w go together");
    for (int j = 0; j < nsrc; ++j)
        if (src[j] < 0 || src[j] >= c->S) return fail(c, XK_EINVAL, "pathways: source %d out of range", src[j]);
    cudaMemcpyAsync(c->path_src, src, sizeof(int) * nsrc, cudaMemcpyHostToDevice, c->st);
    cudaError_t e = launch_pathways(c->col, c->pgraph, q, c->path_w, nsrc, c->path_src, dist, pred_sp, pred_edge,
                                    lim_edge, lim_w, c->st);
    if (e != cudaSuccess) return fail(c, XK_EINVAL, "pathways launch: %s", cudaGetErrorString(e));
    return finish_eval(c, "pathways");
}

// ---------------------------------------------------------------- variable-order BDF

namespace {

// Derivative weights at tau[0] of the Lagrange basis on nodes tau[0..q] (the corrector), and the
// weights of the interpolant through m nodes evaluated at t (the predictors).
void bdf_weights(int q, const double *tau, double *c)
{
    double c0 = 0.0;
    for (int m = 1; m <= q; ++m) c0 += 1.0 / (tau[0] - tau[m]);
    c[0] = c0;
    for (int j = 1; j <= q; ++j) {
        double num = 1.0, den = 1.0;
        for (int m = 0; m <= q; ++m) {
            if (m == j) continue;
            if (m != 0) num *= tau[0] - tau[m];
            den *= tau[j] - tau[m];
        }
        c[j] = num / den;
    }
}

void interp_weights(int m, const double *tau, double t, double *w)
{
    for (int j = 0; j < m; ++j) {
        double v = 1.0;
        for (int i = 0; i < m; ++i)
            if (i != j) v *= (t - tau[i]) / (tau[j] - tau[i]);
        w[j] = v;
    }
}

BdfCombo make_combo(int m, const int *slot, const double *w)
{
    BdfCombo b{};
    b.m = m;
    for (int j = 0; j < m; ++j) {
        b.slot[j] = slot[j];
        b.w[j] = w[j];
    }
    return b;
}

double from_bits(unsigned long long u)
{
    double d;
    std::memcpy(&d, &u, sizeof d);
    return d;
}

}  // namespace

int xk_bdf_run(xk_ctx *c, const xk_bdf_config *cfg, double h0, double t_end, int stop_at_steady, int max_steps,
               xk_bdf_info *info)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!cfg || !info || !(cfg->rtol > 0.0) || cfg->qmax < 1 || cfg->qmax > 5 || !(h0 > 0.0) || !(t_end > 0.0) ||
        max_steps <= 0 || !(cfg->grow >= 1.0))
        return fail(c, XK_EINVAL, "bdf: bad arguments");
    ensure_rates(c);
    const long long N = (long long)c->L * c->S;
    const int HMAX = cfg->qmax + 2, qmax = cfg->qmax;
    const Policy pol = policy_of(c->cfg);
    int slot[kBdfHist];
    for (int j = 0; j < kBdfHist; ++j) slot[j] = j;
    double th[kBdfHist] = {0.0};
    cudaMemcpyAsync(c->bdfY + (size_t)slot[0] * N, c->col.n, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->st);
    std::memset(info, 0, sizeof *info);
    int hist = 1, q = 1, nq = 0, nrej = 0;
    double t = 0.0, h = std::min(h0, t_end);
    const double dto_fp64 = c->cfg.precision == XK_PREC_FP64;
    int status = XK_ENOCONV;
    while (info->steps < max_steps) {
        info->steps++;
        const int qe = std::min(q, hist);
        double tau[kBdfHist], cc[kBdfHist], w[kBdfHist], w1[kBdfHist], w2[kBdfHist];
        tau[0] = t + h;
        for (int j = 1; j <= qe; ++j) tau[j] = th[j - 1];
        bdf_weights(qe, tau, cc);
        const int m = std::min(qe + 1, hist);
        interp_weights(m, th, t + h, w);
        BdfStepArgs a{};
        a.pred = make_combo(m, slot, w);
        a.hist = make_combo(qe, slot, cc + 1);
        a.c0 = cc[0];
        const bool sel = !cfg->fixed_order && nq + 1 >= qe + 1;
        if (sel && qe > 1) {
            interp_weights(qe, th, t + h, w1);
            a.lo = make_combo(qe, slot, w1);
        }
        if (sel && qe < qmax && hist >= qe + 2) {
            interp_weights(qe + 2, th, t + h, w2);
            a.hi = make_combo(qe + 2, slot, w2);
        }
        a.K = qe + 1.0;
        a.Klo = qe;
        a.Khi = qe + 2.0;
        a.rtol = cfg->rtol;
        a.neg_tol = pol.neg_tol;
        a.f_floor = pol.f_floor;
        a.newest = slot[0];
        launch_bdf_predict(N, c->bdfY, a, c->bdf_yhat, c->bdf_g, c->st);
        // the backward-Euler system with dt = 1/c0 and the history terms off the right-hand side
        Ctl init = fresh_ctl(c);
        init.dt = 1.0 / cc[0];
        init.dt_fp64 = 1e300;
        *c->ctl_host = init;
        cudaMemcpyAsync(c->ctl_aux, c->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
        c->col.fshift = c->bdf_g;
        rc = enqueue_linear_step(c, c->bdf_yhat, dto_fp64 ? 1.0 / cc[0] : 0.0, c->bdf_delta, c->ctl_aux);
        c->col.fshift = nullptr;
        if (rc) return rc;
        cudaMemsetAsync(c->bdf_res, 0, sizeof(BdfResult), c->st);
        launch_bdf_check(c->col, c->bdfY, a, c->bdf_yhat, c->bdf_delta, c->bdf_ynew, c->bdf_res, c->st);
        BdfResult res{};
        cudaMemcpyAsync(c->ctl_host, c->ctl_aux, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
        cudaMemcpyAsync(&res, c->bdf_res, sizeof res, cudaMemcpyDeviceToHost, c->st);
        if ((rc = finish_eval(c, "bdf step"))) return rc;
        if (c->ctl_host->err_timeout) return timed_out(c);
        if (c->ctl_host->err_singular) return fail(c, XK_ESINGULAR, "bdf: zero pivot in a diagonal block");
        info->solver_iters += std::max(c->ctl_host->solver_iters, 0);
        const bool bad = res.bad != 0;
        double err = bad ? INFINITY : from_bits(res.err);
        if (cfg->fixed_step) {
            if (bad) return fail(c, XK_ENEG, "bdf: non-finite or negative state at a fixed step");
            err = 0.0;
        }
        if (bad || err > 1.0) {
            info->rejected++;
            nrej++;
            double f = bad ? 0.25 : 0.9 * std::pow(err, -1.0 / (qe + 1));
            if (!bad) f = std::min(0.9, std::max(0.2, f));
            h *= f;
            if (nrej >= 2 && q > 1) {
                q--;
                nq = 0;
            }
            if (h < pol.dt_min) return fail(c, XK_ENEG, "bdf: step %.3g below dt_min", h);
            continue;
        }
        const double relc = from_bits(res.relc);
        double eta = std::pow(std::max(err, 1e-10), -1.0 / (qe + 1)) / 1.2;
        int qnew = q;
        nq++;
        if (!cfg->fixed_order && nq >= qe + 1) {
            if (qe > 1) {
                const double e1 = from_bits(res.err_lo);
                const double eta1 = std::pow(std::max(e1, 1e-10), -1.0 / qe) / 1.3;
                if (eta1 > eta) {
                    eta = eta1;
                    qnew = qe - 1;
                }
            }
            if (qe < qmax && hist >= qe + 2) {
                const double e2 = from_bits(res.err_hi);
                const double eta2 = std::pow(std::max(e2, 1e-10), -1.0 / (qe + 2)) / 1.4;
                if (eta2 > eta) {
                    eta = eta2;
                    qnew = qe + 1;
                }
            }
            if (qnew != q) nq = 0;
        }
        if (cfg->fixed_order > 0) qnew = std::min(cfg->fixed_order, qmax);
        // push: the oldest buffer takes the new state
        const int nb = slot[HMAX - 1];
        for (int j = HMAX - 1; j > 0; --j) {
            slot[j] = slot[j - 1];
            th[j] = th[j - 1];
        }
        slot[0] = nb;
        th[0] = t + h;
        launch_bdf_accept(N, c->bdf_ynew, c->bdfY + (size_t)nb * N, c->col.n, c->st);
        if (hist < HMAX) hist++;
        info->accepted++;
        info->order_steps[qe]++;
        nrej = 0;
        const double hused = h;
        t += h;
        q = qnew;
        if (!cfg->fixed_step) {
            eta = std::min(cfg->grow, std::max(0.2, eta));
            h *= eta;
            h = std::min(h, pol.dt_max);
        }
        info->max_rel = relc;
        if (stop_at_steady && hused >= pol.ss_dt && relc < pol.ss_tol) {
            info->converged = 1;
            status = XK_OK;
            break;
        }
        if (t >= t_end * (1.0 - 1e-12)) {
            status = XK_OK;
            break;
        }
        h = std::min(h, t_end - t);
    }
    info->t = t;
    info->h = h;
    info->q = q;
    if ((rc = finish_eval(c, "bdf run"))) return rc;
    if (status != XK_OK) return fail(c, XK_ENOCONV, "bdf: %d attempts without reaching the end", max_steps);
    return XK_OK;
}

// ---------------------------------------------------------------- Lagrangian parcel scheme

int xk_parcel_begin(xk_ctx *c, int max_visit_steps, double h)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (max_visit_steps <= 0 || !(h > 0.0)) return fail(c, XK_EINVAL, "parcel: bad arguments");
    if (!(c->L >= 1)) return fail(c, XK_EINVAL, "parcel: no layers");
    for (int k = 0; k < c->L; ++k)
        if (!(c->Kzz[k] > 0.0)) return fail(c, XK_EINVAL, "parcel: K_zz must be positive (residence time dz^2 / K_zz)");
    ensure_rates(c);
    // photolysis from the stored profile at the start of the iteration; molecular-only u, v
    launch_photolysis(c->col, c->col.n, c->st);
    cudaMemsetAsync(c->parcel_kzz0, 0, sizeof(double) * c->L, c->st);
    launch_transport_coeffs(c->col, c->parcel_kzz0, const_cast<double *>(c->parcel.um),
                            const_cast<double *>(c->parcel.vm), c->st);
    ParcelState init{};
    init.h = h;
    init.status = -1;
    *c->parcel_host = init;
    cudaMemcpyAsync(c->parcel.st, c->parcel_host, sizeof(ParcelState), cudaMemcpyHostToDevice, c->st);
    ParcelArgs a = c->parcel;
    a.pol = policy_of(c->cfg);
    a.max_visit_steps = max_visit_steps;
    cudaError_t le = launch_parcel_iteration(c->col, a, c->st);
    if (le != cudaSuccess) return fail(c, XK_ECUDA, "parcel launch: %s", cudaGetErrorString(le));
    c->parcel_max_visit = max_visit_steps;
    cudaMemcpyAsync(c->parcel_host, c->parcel.st, sizeof(ParcelState), cudaMemcpyDeviceToHost, c->st);
    return cuda_check(c, "parcel begin");
}

int xk_parcel_end(xk_ctx *c, xk_parcel_info *info)
{
    int rc = need_ready(c);
    if (rc) return rc;
    if (!info) return fail(c, XK_EINVAL, "parcel: null info");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "parcel iteration: %s", cudaGetErrorString(e));
    const ParcelState &h = *c->parcel_host;
    info->h = h.h;
    info->steps = h.steps;
    info->rejected = h.rejected;
    info->max_change = h.max_change;
    if (h.status == XK_ESINGULAR) return fail(c, XK_ESINGULAR, "parcel: singular system at visit %d", h.visit);
    if (h.status == XK_ENEG) return fail(c, XK_ENEG, "parcel: step below dt_min at visit %d", h.visit);
    if (h.status == XK_ENOCONV)
        return fail(c, XK_ENOCONV, "parcel: more than %d steps in visit %d", c->parcel_max_visit, h.visit);
    if (h.status != 0) return fail(c, XK_ECUDA, "parcel: iteration did not complete (status %d)", h.status);
    return XK_OK;
}

int xk_parcel_iteration(xk_ctx *c, int max_visit_steps, xk_parcel_info *info)
{
    if (!info) return c ? fail(c, XK_EINVAL, "parcel: null info") : XK_EINVAL;
    int rc = xk_parcel_begin(c, max_visit_steps, info->h);
    if (rc) return rc;
    return xk_parcel_end(c, info);
}

int xk_parcel_run(xk_ctx *c, int max_visit_steps, int max_iter, double tol, xk_parcel_info *info, int *iterations)
{
    if (!c || !info || !iterations || max_iter <= 0 || !(tol > 0.0)) return c ? fail(c, XK_EINVAL, "parcel run: bad arguments") : XK_EINVAL;
    long long steps = 0, rejected = 0;
    int it = 0, rc = XK_OK;
    while (it < max_iter) {
        rc = xk_parcel_iteration(c, max_visit_steps, info);
        ++it;
        steps += info->steps;
        rejected += info->rejected;
        if (rc != XK_OK || info->max_change < tol) break;
    }
    info->steps = steps;
    info->rejected = rejected;
    *iterations = it;
    if (rc != XK_OK) return rc;
    if (!(info->max_change < tol)) return fail(c, XK_ENOCONV, "parcel: change %.3g after %d iterations", info->max_change, it);
    return XK_OK;
}

int xk_profile(xk_ctx *c, int enable)
{
    if (!c) return XK_EINVAL;
    c->prof = enable != 0;
    for (auto &u : c->ev_used) u = 0;
    return XK_OK;
}

int xk_profile_read(xk_ctx *c, double *ms, long long *calls, int n)
{
    if (!c || n < 0 || (n > 0 && (!ms || !calls))) return XK_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return fail(c, XK_ECUDA, "profile sync: %s", cudaGetErrorString(e));
    for (int p = 0; p < n && p < XK_PH_COUNT; ++p) {
        double tot = 0.0;
        for (size_t i = 0; i < c->ev_used[p]; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, c->ev[p][i].first, c->ev[p][i].second) == cudaSuccess) tot += t;
            else cudaGetLastError();
        }
        ms[p] = tot;
        calls[p] = (long long)c->ev_used[p];
    }
    return XK_OK;
}

}  // extern "C"
