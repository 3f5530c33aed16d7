// Host orchestration of the implicit step behind the C ABI (include/rhi.h): buffers, the
// globalised inexact Newton iteration (Sec. 3.2), the Schur-system CG solve with its
// multigrid preconditioner (Sec. 3.2.1, step (ii)), profiling and statistics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "rhi_linear.cuh"
#include "rhi_mlp.cuh"

using namespace rhi;

namespace {

// ---------------------------------------------------------------------------------------------
// launch hook: counts launches, and with profiling on brackets each one with CUDA events

struct Profiler : LaunchHook {
    cudaStream_t st = nullptr;
    bool on = false;
    int launches = 0;
    std::vector<cudaEvent_t> pool;
    struct Rec { const char* name; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::map<std::string, std::pair<double, int>> acc;
    const char* cur = nullptr;
    cudaEvent_t cur_a = nullptr;

    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    std::vector<std::string> only;     // when non-empty: time only launches of these names
    void begin(const char* name) override {
        ++launches;
        if (!on) return;
        if (!only.empty() && std::find(only.begin(), only.end(), name) == only.end()) return;
        cur = name;
        cur_a = get();
        cudaEventRecord(cur_a, st);
    }
    void end() override {
        if (!on || !cur) return;
        cudaEvent_t b = get();
        cudaEventRecord(b, st);
        pending.push_back({cur, cur_a, b});
        cur = nullptr;
    }
    void resolve() {
        for (auto& r : pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess) cudaEventElapsedTime(&ms, r.a, r.b);
            auto& v = acc[r.name];
            v.first += ms;
            v.second += 1;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    ~Profiler() override {
        for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

template <typename T>
struct Level {
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    T* diag = nullptr;
    T* wid = nullptr;           // omega / diag (smoother)
    T* loc = nullptr;           // diag - the row's six couplings (FP64 restriction; FP32: none)
    T* W[3] = {nullptr, nullptr, nullptr};
    T* Wp[3] = {nullptr, nullptr, nullptr};     // non-symmetric levels only
    T* b = nullptr;
    T* x = nullptr;
    T* xt = nullptr;
};

}  // namespace

struct rhi_ctx {
    rhi_grid grid{};
    rhi_bc bc{};
    rhi_params prm{};
    int ns = 1, nv = 3, nm = 2;
    long long N = 0;
    int per[3] = {0, 0, 0};
    cudaStream_t st = nullptr;
    std::string err;
    rhi_stats stats{};
    Profiler prof;
    bool have_state = false;
    bool have_linear = false;

    std::vector<void*> allocs;

    // state U^n
    double *E_s = nullptr, *e_s = nullptr, *n_s = nullptr, *nH = nullptr, *src = nullptr,
           *Tiso = nullptr;
    // the state before the last accepted step and that step's length (the learned guess's
    // view of the previous change; ionization model only)
    double *E_p = nullptr, *e_p = nullptr, *n_p = nullptr;
    double dt_prev = 0.0;
    bool have_prev = false;
    // two work iterates, contiguous (e_c | n_1 .. | E), their opacity and face coefficients
    double* U[2] = {nullptr, nullptr};
    double* kap[2] = {nullptr, nullptr};
    double* W[2] = {nullptr, nullptr};
    double* PQ[2] = {nullptr, nullptr};         // Newton-matrix face entries (dD/dE kept)
    double* Kf[2] = {nullptr, nullptr};         // exact matrix: (1/2) dW/dkappa dE per face
    double* Upred = nullptr;                    // explicit predictor of the step (dt_norm)
    double* diag_ns[2] = {nullptr, nullptr};
    double* g = nullptr;
    double *diag[2] = {nullptr, nullptr}, *rhs[2] = {nullptr, nullptr};
    double *fMt[2] = {nullptr, nullptr}, *MiU[2] = {nullptr, nullptr};
    double* f_tmp = nullptr;
    // CG
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    // BiCGStab
    double *rh = nullptr, *v = nullptr, *s = nullptr, *t = nullptr, *ph = nullptr, *sh = nullptr;
    double* partials = nullptr;
    double* scal = nullptr;
    double* h_scal = nullptr;   // pinned
    int* d_flag = nullptr;
    double2* table = nullptr;
    // multigrid
    std::vector<Level<double>> mg64;
    std::vector<Level<float>> mg32;
    // the lagged-D Schur matrix, the Newton matrix when dD/dE is kept, and the finest operator
    // the preconditioner was last set up from (one of the two; pc_nonsym: the Newton matrix)
    Op<double> op0{};
    OpNS opns{};
    Op<double> pc0{};
    bool pc_nonsym = false;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    // the FP32 V-cycle captured as a CUDA graph
    struct VGraph {
        cudaGraphExec_t exec = nullptr;
        cudaStream_t st = nullptr;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        double scale = 0.0;
        bool nonsym = false;
        std::vector<float*> post;       // level buffers (x, xt) after the captured cycle
        int kernels = 0;
        bool failed = false;
    } vg;

    // the BiCGStab solve as one CUDA graph (a while node whose body is one iteration),
    // cached per set of buffers and operator scale
    struct KGraph {
        const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        double scale = 0.0;
        bool nonsym = false;
        cudaGraphExec_t exec = nullptr;
        int k_init = 0, k_body = 0;
    };
    std::vector<KGraph> kg;
    cudaStream_t kst = nullptr;           // capture stream
    bool kg_failed = false;
    double* h_ctl = nullptr;              // pinned: S_THR, S_MAXIT, S_INNER of the next solve
    int* h_kerr = nullptr;                // pinned: the staged multigrid sweep's wait flag
    int host_syncs = 0;                   // blocking device-to-host reads of the last step
    int kg_body_kernels = 0;              // kernels per iteration of the last graph solve

    // learned guess: FP32 master weights, Adam moments, gradient, BF16 inference copy;
    // scratch of the training / inspection entry points grows on demand
    float *mlp_w = nullptr, *mlp_m1 = nullptr, *mlp_m2 = nullptr, *mlp_g = nullptr;
    MlpPacked* mlp_pk = nullptr;
    bool mlp_ready = false;
    long long mlp_t = 0;                  // Adam steps taken
    int mlp_skip = 0;                     // steps left that skip the network (mlp_retry)
    struct Scratch { void* p = nullptr; size_t bytes = 0; };
    Scratch mlp_scr[6];                   // act, del, partials, X, Y, grad staging
    ~rhi_ctx() { for (auto& s : mlp_scr) if (s.p) cudaFree(s.p); }
};

namespace {

int fail(rhi_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(h, RHI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int dalloc(rhi_ctx* h, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return fail(h, RHI_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->allocs.push_back(v);
    *p = (T*)v;
    return RHI_OK;
}

StepParams make_params(const rhi_ctx* h, double dt, double a, double adot) {
    StepParams P{};
    P.nx = h->grid.nx; P.ny = h->grid.ny; P.nz = h->grid.nz;
    P.fd_nx = make_fastdiv((unsigned)P.nx);
    P.fd_nxy = make_fastdiv((unsigned)P.nx * (unsigned)P.ny);
    P.N = h->N;
    P.per_x = h->per[0]; P.per_y = h->per[1]; P.per_z = h->per[2];
    P.dir_mask = 0;
    for (int d = 0; d < 6; ++d) {
        P.Eb[d] = h->bc.value[d];
        if (h->bc.kind[d] == RHI_BC_DIRICHLET) P.dir_mask |= 1 << d;
    }
    P.dx = h->grid.dx;
    P.a = a; P.ia3 = 1.0 / (a * a * a); P.adot_a = adot / a;
    P.dt = dt; P.dth = dt * h->prm.theta; P.dtm1 = dt * (h->prm.theta - 1.0);
    P.inv_adx = 1.0 / (a * h->grid.dx);
    P.half_adx = 0.5 * a * h->grid.dx;
    P.inv_a2dx2 = P.inv_adx * P.inv_adx;
    const int nmax = std::max(h->grid.nx, std::max(h->grid.ny, h->grid.nz));
    P.R_min = 1.0 / (a * nmax * h->grid.dx);
    P.kappa_floor = h->prm.kappa_floor;
    P.m_grey = (double)h->prm.m_grey;
    P.isothermal = h->prm.isothermal; P.limiter = h->prm.limiter;
    P.limiter_newton = h->prm.limiter_jacobian;
    P.y_he = h->prm.y_he;
    P.u_e = h->prm.u_e; P.u_n = h->prm.u_n; P.u_E = h->prm.u_E;
    P.iu_e = 1.0 / P.u_e; P.iu_n = 1.0 / P.u_n; P.iu_E = 1.0 / P.u_E;
    P.sc_ne = P.dth * P.u_n * P.iu_e;
    P.sc_en = P.dth * P.u_e * P.iu_n;
    P.sc_Ee = P.dth * P.u_E * P.iu_e;
    P.sc_En = P.dth * P.u_E * P.iu_n;
    P.sc_eE = P.dth * P.u_e * P.iu_E;
    P.sc_nE = P.dth * P.u_n * P.iu_E;
    for (int X = 0; X < 3; ++X) { P.sk[X] = h->prm.sk[X]; P.pg[X] = h->prm.pgam[X]; P.ph[X] = h->prm.ph[X]; }
    P.tau = h->prm.tau;
    P.lte = h->prm.model == RHI_MODEL_LTE;
    P.kappa_total = h->prm.kappa_total;
    P.kappa_planck = h->prm.kappa_planck;
    P.lte_cT = (GAMMA - 1.0) * h->prm.mu * M_H / K_BOLTZ;
    P.table = h->table;
    return P;
}

// names of the physics kernels for the profiler
struct Scope {
    Profiler& p;
    Scope(Profiler& pr, const char* n) : p(pr) { p.begin(n); }
    ~Scope() { p.end(); }
};

int read_scalar(rhi_ctx* h, int slot, double* out) {
    CK(cudaMemcpyAsync(h->h_scal, h->scal, sizeof(double) * S_NSCAL, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->host_syncs += 1;
    *out = h->h_scal[slot];
    return RHI_OK;
}

// ||f||_RMS from the cell kernel's partials
int residual_norm(rhi_ctx* h, int nparts, double* out) {
    LinLaunch L(h->st, &h->prof);
    CK(L.reduce(h->partials, nparts, h->scal, RED_SUM, S_TMP));
    double s;
    int rc = read_scalar(h, S_TMP, &s);
    if (rc) return rc;
    *out = std::sqrt(s / ((double)h->N * h->nv));
    return RHI_OK;
}

// ---------------------------------------------------------------------------------------------
// multigrid

void level_dims(int n, int& c) { c = (n + 1) / 2; }

int mg_build_levels(rhi_ctx* h) {
    const int L = std::max(1, h->prm.mg_levels);
    int nx = h->grid.nx, ny = h->grid.ny, nz = h->grid.nz;
    std::vector<int> dims;
    for (int l = 0; l < L; ++l) {
        dims.push_back(nx); dims.push_back(ny); dims.push_back(nz);
        if (nx == 1 && ny == 1 && nz == 1) break;
        int cx, cy, cz;
        level_dims(nx, cx); level_dims(ny, cy); level_dims(nz, cz);
        nx = cx; ny = cy; nz = cz;
    }
    const int nl = (int)dims.size() / 3;
    // the hierarchy of the non-symmetric Newton matrix carries a second face array per axis
    const bool nonsym = h->prm.mg_matrix == 1 && h->prm.limiter_jacobian != 0;
    if (h->prm.precond == RHI_PRECOND_MG_FP64) {
        h->mg64.resize(nl);
        for (int l = 0; l < nl; ++l) {
            auto& v = h->mg64[l];
            v.nx = dims[3 * l]; v.ny = dims[3 * l + 1]; v.nz = dims[3 * l + 2];
            v.N = (long long)v.nx * v.ny * v.nz;
            int rc;
            if (l > 0) {
                if ((rc = dalloc(h, &v.diag, v.N))) return rc;
                for (int a = 0; a < 3; ++a) if ((rc = dalloc(h, &v.W[a], v.N))) return rc;
                if (nonsym)
                    for (int a = 0; a < 3; ++a) if ((rc = dalloc(h, &v.Wp[a], v.N))) return rc;
                if ((rc = dalloc(h, &v.b, v.N))) return rc;
                if ((rc = dalloc(h, &v.x, v.N))) return rc;
            }
            if ((rc = dalloc(h, &v.xt, v.N))) return rc;
            if ((rc = dalloc(h, &v.wid, v.N))) return rc;
            if ((rc = dalloc(h, &v.loc, v.N))) return rc;
        }
    } else if (h->prm.precond == RHI_PRECOND_MG_FP32) {
        h->mg32.resize(nl);
        for (int l = 0; l < nl; ++l) {
            auto& v = h->mg32[l];
            v.nx = dims[3 * l]; v.ny = dims[3 * l + 1]; v.nz = dims[3 * l + 2];
            v.N = (long long)v.nx * v.ny * v.nz;
            int rc;
            if ((rc = dalloc(h, &v.diag, v.N))) return rc;
            if ((rc = dalloc(h, &v.wid, v.N))) return rc;
            for (int a = 0; a < 3; ++a) if ((rc = dalloc(h, &v.W[a], v.N))) return rc;
            if (nonsym)
                for (int a = 0; a < 3; ++a) if ((rc = dalloc(h, &v.Wp[a], v.N))) return rc;
            if ((rc = dalloc(h, &v.b, v.N))) return rc;
            if ((rc = dalloc(h, &v.x, v.N))) return rc;
            if ((rc = dalloc(h, &v.xt, v.N))) return rc;
        }
    }
    return RHI_OK;
}

template <typename T>
Op<T> level_op(const rhi_ctx* h, const Level<T>& v) {
    Op<T> A{};
    A.nx = v.nx; A.ny = v.ny; A.nz = v.nz; A.N = v.N;
    A.fd_nx = make_fastdiv((unsigned)v.nx);
    A.fd_nxy = make_fastdiv((unsigned)v.nx * (unsigned)v.ny);
    for (int a = 0; a < 3; ++a) {
        A.per[a] = h->per[a];
        A.W[a] = v.W[a];
        A.Wp[a] = h->pc_nonsym && v.Wp[a] ? v.Wp[a] : v.W[a];
    }
    A.diag = v.diag;
    A.wid = v.wid;
    A.loc = v.loc;
    A.scale = T(1);
    return A;
}

// the Newton matrix that keeps dD/dE (h->opns) as a multigrid operator: W = Q, Wp = P
Op<double> newton_op(const rhi_ctx* h) {
    const OpNS& B = h->opns;
    Op<double> A{};
    A.nx = B.nx; A.ny = B.ny; A.nz = B.nz; A.N = B.N;
    A.fd_nx = B.fd_nx; A.fd_nxy = B.fd_nxy;
    for (int a = 0; a < 3; ++a) { A.per[a] = B.per[a]; A.W[a] = B.Q[a]; A.Wp[a] = B.P[a]; }
    A.diag = B.diag;
    A.scale = B.scale;
    return A;
}

// coarse operators for the finest operator A0 (the lagged-D matrix h->op0, or the Newton matrix
// when nonsym); A0 becomes the preconditioner's finest operator h->pc0
int precond_setup(rhi_ctx* h, const Op<double>& A0, bool nonsym) {
    LinLaunch L(h->st, &h->prof);
    const double om = h->prm.mg_omega;
    h->pc0 = A0;
    h->pc_nonsym = nonsym;
    if (h->prm.precond == RHI_PRECOND_MG_FP64) {
        auto& lv = h->mg64;
        if (nonsym && lv.size() > 1 && !lv[1].Wp[0])
            return fail(h, RHI_ERR_ARG, "multigrid of the Newton matrix needs params.mg_matrix = 1");
        h->pc0.wid = lv[0].wid;
        h->pc0.loc = lv[0].loc;
        CK((L.level_prep<double, double>(h->pc0, om, lv[0].wid, lv[0].loc)));
        for (size_t l = 0; l + 1 < lv.size(); ++l) {
            Op<double> A = (l == 0) ? h->pc0 : level_op(h, lv[l]);
            auto& c = lv[l + 1];
            CK((L.coarsen<double, double>(A, c.nx, c.ny, c.nz, c.diag, c.W, nonsym ? c.Wp : nullptr)));
            CK(L.diag_faces<double>(level_op(h, c), c.diag));
            CK((L.level_prep<double, double>(level_op(h, c), om, c.wid, c.loc)));
        }
    } else if (h->prm.precond == RHI_PRECOND_MG_FP32) {
        auto& lv = h->mg32;
        if (nonsym && !lv[0].Wp[0])
            return fail(h, RHI_ERR_ARG, "multigrid of the Newton matrix needs params.mg_matrix = 1");
        CK(L.cast_op(h->pc0, lv[0].diag, lv[0].W, nonsym ? lv[0].Wp : nullptr));
        // the finest level's omega / diag from the FP64 operator (the FP32 restriction takes
        // each child's full row and needs no local part)
        CK((L.level_prep<double, float>(h->pc0, om, lv[0].wid, nullptr)));
        for (size_t l = 0; l + 1 < lv.size(); ++l) {
            auto& c = lv[l + 1];
            if (l == 0)
                CK((L.coarsen<double, float>(h->pc0, c.nx, c.ny, c.nz, c.diag, c.W, nonsym ? c.Wp : nullptr)));
            else
                CK((L.coarsen<float, float>(level_op(h, lv[l]), c.nx, c.ny, c.nz, c.diag, c.W, nonsym ? c.Wp : nullptr)));
            CK(L.diag_faces<float>(level_op(h, c), c.diag));
            CK((L.level_prep<float, float>(level_op(h, c), om, c.wid, nullptr)));
        }
    }
    return RHI_OK;
}

// the preconditioner of the system the Krylov method solves: the Newton matrix's own
// hierarchy when params.mg_matrix = 1 and the matrix keeps dD/dE, else the lagged-D matrix's
int precond_setup_newton(rhi_ctx* h) {
    const bool nonsym = h->prm.mg_matrix == 1 && h->prm.limiter_jacobian != 0 &&
                        h->prm.precond != RHI_PRECOND_JACOBI;
    return precond_setup(h, nonsym ? newton_op(h) : h->op0, nonsym);
}

// one V-cycle on levels l.. with right-hand side lv[l].b; result in lv[l].x
template <typename T>
int vcycle(rhi_ctx* h, std::vector<Level<T>>& lv, size_t l, const Op<T>& A0,
           cudaStream_t st = nullptr, LaunchHook* hook = nullptr, const double* skip = nullptr) {
    if (!hook) { st = h->st; hook = &h->prof; }
    LinLaunch L(st, hook);
    L.fine_N = h->N;
    L.skip = skip;
    Level<T>& v = lv[l];
    const Op<T> A = (l == 0) ? A0 : level_op(h, v);
    const T om = (T)h->prm.mg_omega;
    if (l + 1 == lv.size()) {
        if (v.N <= COARSE_MAX) {
            // all sweeps in one launch; x and xt alternate as in the loop below
            CK(L.coarse_solve<T>(A, v.b, v.x, v.xt, om, h->prm.mg_coarse_sweeps));
            if ((h->prm.mg_coarse_sweeps - 1) % 2) std::swap(v.x, v.xt);
            return RHI_OK;
        }
        CK(L.smooth<T>(A, v.b, v.x, v.x, om, 1));
        for (int s = 1; s < h->prm.mg_coarse_sweeps; ++s) {
            CK(L.smooth<T>(A, v.b, v.x, v.xt, om, 0));
            std::swap(v.x, v.xt);
        }
        return RHI_OK;
    }
    CK(L.smooth<T>(A, v.b, v.x, v.x, om, 1));
    for (int s = 1; s < h->prm.mg_pre; ++s) {
        CK(L.smooth<T>(A, v.b, v.x, v.xt, om, 0));
        std::swap(v.x, v.xt);
    }
    Level<T>& c = lv[l + 1];
    CK(L.restrict_res<T>(A, v.b, v.x, c.nx, c.ny, c.nz, c.b));
    int rc = vcycle<T>(h, lv, l + 1, A0, st, hook, skip);
    if (rc) return rc;
    // (a sweep that reads the coarse correction on the fly measured 3.6x slower than the
    // separate prolongation and sweep at 256^3, so the two stay separate)
    CK(L.prolong<T>(v.nx, v.ny, v.nz, c.nx, c.ny, c.x, v.x));
    for (int s = 0; s < h->prm.mg_post; ++s) {
        CK(L.smooth<T>(A, v.b, v.x, v.xt, om, 0));
        std::swap(v.x, v.xt);
    }
    return RHI_OK;
}

// ---- the FP32 V-cycle as a CUDA graph
//
// One V-cycle is about 45 launches, most of them on grids of 64^3 cells and below, where the
// launch gap is longer than the kernel.  The cycle is captured once (on a private stream) and
// replayed as one graph launch ordered after / before the handle's stream by events.  The
// graph binds the level buffers and the operator's scale (dt theta) at capture; it is
// captured again when the scale changes or the host's view of the ping-pong buffers no longer
// matches the state after capture (a direct V-cycle ran in between).

struct Counter : LaunchHook {
    int n = 0;
    void begin(const char*) override { ++n; }
    void end() override {}
};

bool vcycle_graph_usable(const rhi_ctx* h) {
    if (!h->prm.vcycle_graph || h->vg.failed) return false;
    if (!h->prof.on) return true;
    // per-launch timing of a V-cycle kernel needs the direct launches
    if (h->prof.only.empty()) return false;
    for (const auto& nm : h->prof.only)
        if (nm.compare(0, 3, "mg_") == 0) return false;
    return true;
}

int vcycle_graph(rhi_ctx* h, const Op<float>& A0) {
    auto& lv = h->mg32;
    auto& g = h->vg;
    bool valid = g.exec && g.scale == (double)A0.scale && g.nonsym == h->pc_nonsym &&
                 g.post.size() == 2 * lv.size();
    for (size_t l = 0; valid && l < lv.size(); ++l)
        valid = g.post[2 * l] == lv[l].x && g.post[2 * l + 1] == lv[l].xt;
    if (!valid) {
        if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
        if (!g.st) {
            CK(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&g.ev0, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&g.ev1, cudaEventDisableTiming));
        }
        Counter cnt;
        CK(cudaStreamBeginCapture(g.st, cudaStreamCaptureModeThreadLocal));
        int rc = vcycle<float>(h, lv, 0, A0, g.st, &cnt);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(g.st, &graph);
        if (rc || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            g.failed = true;
            return rc ? rc : fail(h, RHI_ERR_CUDA, std::string("V-cycle capture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.failed = true;
            g.exec = nullptr;
            return fail(h, RHI_ERR_CUDA, std::string("V-cycle graph: ") + cudaGetErrorString(e));
        }
        g.kernels = cnt.n;
        g.scale = (double)A0.scale;
        g.nonsym = h->pc_nonsym;
        g.post.clear();
        for (auto& v : lv) { g.post.push_back(v.x); g.post.push_back(v.xt); }
    }
    Scope s(h->prof, "mg_vcycle_graph");
    CK(cudaEventRecord(g.ev0, h->st));
    CK(cudaStreamWaitEvent(g.st, g.ev0, 0));
    CK(cudaGraphLaunch(g.exec, g.st));
    CK(cudaEventRecord(g.ev1, g.st));
    CK(cudaStreamWaitEvent(h->st, g.ev1, 0));
    h->prof.launches += g.kernels - 1;      // the scope counted one
    return RHI_OK;
}

// z = M^-1 r, and r.z into the partials; returns the partial count
int precond_apply(rhi_ctx* h, const double* r, double** zout, int& nparts) {
    LinLaunch L(h->st, &h->prof);
    const long long N = h->N;
    if (h->prm.precond == RHI_PRECOND_JACOBI) {
        CK(L.jacobi_dot(N, r, h->pc0.diag, h->z, h->partials, nparts));
        *zout = h->z;
    } else if (h->prm.precond == RHI_PRECOND_MG_FP64) {
        auto& lv = h->mg64;
        lv[0].b = const_cast<double*>(r);
        lv[0].x = h->z;
        int rc = vcycle<double>(h, lv, 0, h->pc0);
        if (rc) return rc;
        // the result may sit in either level-0 buffer
        double* R = lv[0].x;
        if (R != h->z) { lv[0].xt = h->z; h->z = R; }
        *zout = h->z;
        lv[0].x = nullptr;
        CK(L.dot(N, r, h->z, h->partials, nparts));
    } else {
        auto& lv = h->mg32;
        CK(L.to_f32(N, r, lv[0].b));
        Op<float> A0 = level_op(h, lv[0]);
        int rc = vcycle_graph_usable(h) ? vcycle_graph(h, A0) : vcycle<float>(h, lv, 0, A0);
        if (rc) return rc;
        CK(L.from_f32_dot(N, lv[0].x, r, h->z, h->partials, nparts));
        *zout = h->z;
    }
    h->stats.vcycles += 1;
    return RHI_OK;
}

// CG on S sE = rhs to ||r||_RMS <= tol; solution in h->x
int pcg(rhi_ctx* h, const double* rhs, double tol, int* its_out) {
    LinLaunch L(h->st, &h->prof);
    const long long N = h->N;
    const double norm = 1.0 / ((double)N * h->nv);
    int np = 0;
    CK(cudaMemsetAsync(h->scal + S_BREAK, 0, sizeof(double), h->st));     // clear an old breakdown
    CK(L.cg_init(N, rhs, h->r, h->x, h->partials, np));
    CK(L.reduce(h->partials, np, h->scal, RED_SUM, S_RR));
    double rr;
    int rc = read_scalar(h, S_RR, &rr);
    if (rc) return rc;
    int its = 0;
    if (std::sqrt(rr * norm) > tol) {
        double* z = nullptr;
        if ((rc = precond_apply(h, h->r, &z, np))) return rc;
        CK(L.reduce(h->partials, np, h->scal, RED_SUM, S_RZ));
        CK(L.cg_p(N, h->scal, z, h->p, 1));
        for (its = 1; its <= h->prm.max_pcg; ++its) {
            CK(L.matvec_dot(h->op0, h->p, h->q, h->partials, np));
            CK(L.reduce(h->partials, np, h->scal, RED_ALPHA, 0));
            CK(L.cg_xr(N, h->scal, h->x, h->r, h->p, h->q, h->partials, np));
            CK(L.reduce(h->partials, np, h->scal, RED_SUM, S_RR));
            if ((rc = read_scalar(h, S_RR, &rr))) return rc;
            if (h->h_scal[S_BREAK] != 0.0 || !std::isfinite(rr))
                return fail(h, RHI_ERR_NONPHYSICAL, "CG breakdown: p.Sp <= 0 or non-finite residual");
            if (std::sqrt(rr * norm) <= tol) break;
            if ((rc = precond_apply(h, h->r, &z, np))) return rc;
            CK(L.reduce(h->partials, np, h->scal, RED_BETA, 0));
            CK(L.cg_p(N, h->scal, z, h->p, 0));
        }
        if (its > h->prm.max_pcg) its = h->prm.max_pcg;
    }
    *its_out = its;
    return RHI_OK;
}

// M^-1 r into dest with the launcher's stream, hook and skip flag (the second half of a
// BiCGStab iteration); the V-cycle's kernels are launched one by one (also while a graph is
// being captured)
int precond_into(rhi_ctx* h, LinLaunch& L, const double* r, double* dest) {
    const long long N = h->N;
    if (h->prm.precond == RHI_PRECOND_JACOBI) {
        int np = 0;
        CK(L.jacobi_dot(N, r, h->pc0.diag, dest, h->partials, np));
    } else if (h->prm.precond == RHI_PRECOND_MG_FP64) {
        auto& lv = h->mg64;
        double* xt0 = lv[0].xt;
        lv[0].b = const_cast<double*>(r);
        lv[0].x = dest;
        int rc = vcycle<double>(h, lv, 0, h->pc0, L.st, L.hook, L.skip);
        if (rc) return rc;
        if (lv[0].x != dest) CK(L.copy(N, lv[0].x, dest));     // odd number of swaps
        lv[0].x = nullptr;
        lv[0].xt = xt0;
    } else {
        auto& lv = h->mg32;
        CK(L.to_f32(N, r, lv[0].b));
        int rc = vcycle<float>(h, lv, 0, level_op(h, lv[0]), L.st, L.hook, L.skip);
        if (rc) return rc;
        CK(L.from_f32(N, lv[0].x, dest));
    }
    return RHI_OK;
}

// r = b, rh = b, x = 0 and the loop's start (S_RR = S_RHO = r.r, counters cleared)
int bicg_start(rhi_ctx* h, LinLaunch& L, const double* rhs, unsigned long long cond) {
    int np = 0;
    L.skip = nullptr;
    CK(L.bicg_init(h->N, rhs, h->r, h->rh, h->x, h->partials, np));
    CK(L.reduce_loop(h->partials, np, h->scal, RED_BICG_START, cond));
    return RHI_OK;
}

// One iteration of right-preconditioned BiCGStab on the Newton matrix h->opns with every
// decision on the device: p, M^-1 p, v = A M^-1 p, alpha, s and its convergence test; then,
// skipped when s has converged or a breakdown occurred, M^-1 s, t = A M^-1 s and omega; the x /
// r update; the next rho, beta and the continue flag (cond: the graph's while handle, or 0).
int bicg_iteration(rhi_ctx* h, LinLaunch& L, unsigned long long cond) {
    const long long N = h->N;
    int np = 0, rc;
    L.skip = nullptr;
    CK(L.bicg_p(N, h->scal, h->r, h->v, h->p, -1, h->rh));
    if ((rc = precond_into(h, L, h->p, h->ph))) return rc;
    CK(L.matvec_ns(h->opns, h->ph, h->v, h->rh, 0, h->partials, np));
    CK(L.reduce(h->partials, np, h->scal, RED_BICG_ALPHA, 0));
    CK(L.bicg_s(N, h->scal, h->r, h->v, h->s, h->partials, np));
    CK(L.reduce_loop(h->partials, np, h->scal, RED_BICG_SS, 0));
    L.skip = h->scal + S_DONE;
    if ((rc = precond_into(h, L, h->s, h->sh))) return rc;
    CK(L.matvec_ns(h->opns, h->sh, h->t, h->s, 1, h->partials, np));
    CK(L.reduce(h->partials, np, h->scal, RED_BICG_OMEGA, 0));
    L.skip = nullptr;
    CK(L.bicg_xr_loop(N, h->scal, h->x, h->ph, h->sh, h->s, h->t, h->r, h->rh, h->partials, np));
    CK(L.reduce_loop(h->partials, np, h->scal, RED_BICG_NEXT, cond));
    return RHI_OK;
}

// the solve's graph is used unless per-launch timing of one of its kernels is requested
bool krylov_graph_usable(const rhi_ctx* h) {
    if (!h->prm.krylov_graph || h->kg_failed) return false;
    if (!h->prof.on) return true;
    if (h->prof.only.empty()) return false;
    for (const auto& nm : h->prof.only)
        if (nm.compare(0, 3, "mg_") == 0 || nm.compare(0, 5, "bicg_") == 0 || nm == "reduce" ||
            nm == "copy" || nm == "precond_jacobi")
            return false;
    return true;
}

// Captures the whole solve: the start kernels, then a while node (default 1, reset at every
// launch) whose body is one iteration; the last kernel of the start and of each iteration
// writes the node's condition.  The body graph is filled by a second capture.
int krylov_graph_build(rhi_ctx* h, const double* rhs, rhi_ctx::KGraph& g) {
    if (!h->kst) CK(cudaStreamCreateWithFlags(&h->kst, cudaStreamNonBlocking));
    Counter cnt;
    LinLaunch L(h->kst, &cnt);
    L.fine_N = h->N;
    cudaGraph_t graph = nullptr, body = nullptr;
    cudaGraphConditionalHandle hc = 0;
    cudaStreamCaptureStatus stt;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    auto abort_capture = [&](const char* what, cudaError_t e) {
        cudaGraph_t tmp = nullptr;
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(h->kst, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(h->kst, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        if (graph && graph != tmp) cudaGraphDestroy(graph);
        cudaGetLastError();
        h->kg_failed = true;
        return fail(h, RHI_ERR_CUDA, std::string("Krylov graph: ") + what + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaStreamBeginCapture(h->kst, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return abort_capture("begin capture", e);
    e = cudaStreamGetCaptureInfo(h->kst, &stt, nullptr, &graph, &deps, nullptr, &nd);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return abort_capture("conditional handle", e);
    int rc = bicg_start(h, L, rhs, (unsigned long long)hc);
    if (rc) { abort_capture("start kernels", cudaGetLastError()); return rc; }
    e = cudaStreamGetCaptureInfo(h->kst, &stt, nullptr, &graph, &deps, nullptr, &nd);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wn, graph, deps, nullptr, nd, &cp);
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(h->kst, &wn, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return abort_capture("while node", e);
    e = cudaStreamEndCapture(h->kst, &graph);
    if (e != cudaSuccess || !graph) return abort_capture("end capture", e);
    const int k_init = cnt.n;
    body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(h->kst, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return abort_capture("begin body capture", e);
    rc = bicg_iteration(h, L, (unsigned long long)hc);
    if (rc) { abort_capture("body kernels", cudaGetLastError()); return rc; }
    e = cudaStreamEndCapture(h->kst, &body);
    if (e != cudaSuccess) return abort_capture("end body capture", e);
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    graph = nullptr;
    if (e != cudaSuccess) { g.exec = nullptr; return abort_capture("instantiate", e); }
    g.k_init = k_init;
    g.k_body = cnt.n - k_init;
    return RHI_OK;
}

// the outcome of the last BiCGStab solve from the host copy of the scalars (h->h_scal, filled
// by the read that followed the solve): iterations, multigrid cycles, breakdown
int bicg_outcome(rhi_ctx* h, int* its_out) {
    const int its = (int)h->h_scal[S_ITS];
    *its_out = its;
    h->stats.krylov_stalls += h->h_scal[S_STALL] != 0.0 ? 1 : 0;
    h->prof.launches += its * h->kg_body_kernels;
    h->kg_body_kernels = 0;
    if (h->prm.precond != RHI_PRECOND_JACOBI)
        h->stats.vcycles += 2 * its - (h->h_scal[S_HALF] != 0.0 ? 1 : 0);
    if (h->h_scal[S_BREAK] != 0.0 || !std::isfinite(h->h_scal[S_RR]))
        return fail(h, RHI_ERR_NONPHYSICAL, "BiCGStab breakdown");
    return RHI_OK;
}

// Right-preconditioned BiCGStab on the non-symmetric Schur matrix h->opns (dD/dE kept), to
// ||r||_RMS <= tol (counted over the N (N_s + 2) unknowns of eq. rmsnorm); solution in h->x.
// The iteration's control runs on the device: as one CUDA graph launch per solve, or, while
// per-launch timing is on, as direct launches with one host read per iteration.  With
// `deferred` and the graph, the call only enqueues the solve (*its_out = -1): the next host
// read of the scalars brings its outcome back for bicg_outcome.  Otherwise the outcome is read
// here; RHI_ERR_NONPHYSICAL on a breakdown.
int bicgstab(rhi_ctx* h, const double* rhs, double tol, int* its_out, bool deferred = false) {
    const long long N = h->N;
    h->h_ctl[0] = tol * tol * (double)N * h->nv;                   // S_THR: bound on r.r
    h->h_ctl[1] = (double)h->prm.max_pcg;                           // S_MAXIT
    // S_INNER: a restart each time ||r|| falls below krylov_restart of its value at the start.
    // With the FP32 preconditioner, whose rounding slowly erodes the bi-orthogonality, every
    // hundredfold reduction by default; with FP64 only on stagnation.
    double kr = h->prm.krylov_restart;
    if (kr < 0.0) kr = h->prm.precond == RHI_PRECOND_MG_FP32 ? 1e-2 : 0.0;
    h->h_ctl[2] = kr * kr;
    CK(cudaMemcpyAsync(h->scal + S_THR, h->h_ctl, 3 * sizeof(double), cudaMemcpyHostToDevice, h->st));
    int rc = RHI_OK;
    if (krylov_graph_usable(h)) {
        const void* key[6] = {rhs, h->opns.diag, h->opns.P[0], h->pc0.diag, h->pc0.W[0],
                              (const void*)(long long)h->prm.precond};
        rhi_ctx::KGraph* g = nullptr;
        for (auto& c : h->kg)
            if (std::equal(key, key + 6, c.key) && c.scale == h->opns.scale && c.nonsym == h->pc_nonsym)
                g = &c;
        if (!g) {
            if (h->kg.size() >= 8) {
                for (auto& c : h->kg) if (c.exec) cudaGraphExecDestroy(c.exec);
                h->kg.clear();
            }
            rhi_ctx::KGraph ng;
            std::copy(key, key + 6, ng.key);
            ng.scale = h->opns.scale;
            ng.nonsym = h->pc_nonsym;
            if ((rc = krylov_graph_build(h, rhs, ng))) return rc;
            h->kg.push_back(ng);
            g = &h->kg.back();
        }
        {
            Scope s(h->prof, "krylov_graph");
            CK(cudaGraphLaunch(g->exec, h->st));
        }
        // launches: the start kernels now, the iterations' when the count is read back
        h->prof.launches += g->k_init - 1;              // the scope counted one
        h->kg_body_kernels = g->k_body;
        if (deferred) {
            *its_out = -1;
            return RHI_OK;
        }
        double dummy;
        if ((rc = read_scalar(h, S_ITS, &dummy))) return rc;
    } else {
        h->kg_body_kernels = 0;                         // direct launches count themselves
        LinLaunch L(h->st, &h->prof);
        L.fine_N = N;
        if ((rc = bicg_start(h, L, rhs, 0))) return rc;
        double cont = 0.0;
        if ((rc = read_scalar(h, S_CONT, &cont))) return rc;
        while (cont != 0.0) {
            if ((rc = bicg_iteration(h, L, 0))) return rc;
            if ((rc = read_scalar(h, S_CONT, &cont))) return rc;
        }
    }
    return bicg_outcome(h, its_out);
}

// ---------------------------------------------------------------------------------------------
// the physics launches, bracketed for the profiler

PhysBuffers state_buffers(rhi_ctx* h) {
    PhysBuffers B{};
    B.E_n = h->E_s; B.n_n = h->n_s; B.eh = h->e_s; B.nH = h->nH; B.src = h->src; B.Tiso = h->Tiso;
    B.g = h->g;
    B.partials = h->partials;
    return B;
}

int cell(rhi_ctx* h, const StepParams& P, int mode, PhysBuffers B) {
    const int nb = (int)((h->N + cell_block_size() - 1) / cell_block_size());
    Scope s(h->prof, mode == MODE_ITER ? "cell_residual_schur" :
                     mode == MODE_RESID ? "cell_residual" :
                     (mode == MODE_PREP ? "cell_prep_residual_schur" : "cell_prep_predictor"));
    CK(launch_cell(P, h->ns, mode, B, nb, h->st));
    return RHI_OK;
}
int ncell_blocks(const rhi_ctx* h) { return (int)((h->N + cell_block_size() - 1) / cell_block_size()); }

int faces(rhi_ctx* h, const StepParams& P, const double* E, const double* kap, int b) {
    Scope s(h->prof, "faces_limiter");
    CK(launch_faces(P, E, kap, h->W[b], h->PQ[b], h->Kf[b], h->st));
    return RHI_OK;
}
// W alone (an iterate evaluated for its residual only)
int faces_w(rhi_ctx* h, const StepParams& P, const double* E, const double* kap, int b) {
    Scope s(h->prof, "faces_w");
    CK(launch_faces_w(P, h->prm.limiter_jacobian, E, kap, h->W[b], h->st));
    return RHI_OK;
}
// exact Newton matrix: fold the opacity coupling into Schur set `set` built from buffer b
int schur_kappa(rhi_ctx* h, const StepParams& P, int b, int set) {
    if (h->prm.limiter_jacobian != 2) return RHI_OK;
    Scope s(h->prof, "schur_kappa");
    CK(launch_schur_kappa(P, h->ns, h->Kf[b], h->fMt[set], h->MiU[set], h->PQ[b], h->diag_ns[set],
                          h->rhs[set], h->st));
    return RHI_OK;
}
int kappa(rhi_ctx* h, const StepParams& P, const double* n, double* kap) {
    Scope s(h->prof, "kappa");
    CK(launch_kappa(P, h->ns, n, kap, h->st));
    return RHI_OK;
}

void set_op0(rhi_ctx* h, const StepParams& P, int set, const double* W) {
    Op<double>& A = h->op0;
    A.nx = h->grid.nx; A.ny = h->grid.ny; A.nz = h->grid.nz; A.N = h->N;
    A.fd_nx = make_fastdiv((unsigned)A.nx);
    A.fd_nxy = make_fastdiv((unsigned)A.nx * (unsigned)A.ny);
    for (int a = 0; a < 3; ++a) { A.per[a] = h->per[a]; A.W[a] = A.Wp[a] = W + a * h->N; }
    A.diag = h->diag[set];
    A.scale = P.dth;
}

void set_opns(rhi_ctx* h, const StepParams& P, int set, const double* PQ) {
    OpNS& A = h->opns;
    A.nx = h->grid.nx; A.ny = h->grid.ny; A.nz = h->grid.nz; A.N = h->N;
    A.fd_nx = make_fastdiv((unsigned)A.nx);
    A.fd_nxy = make_fastdiv((unsigned)A.nx * (unsigned)A.ny);
    for (int a = 0; a < 3; ++a) {
        A.per[a] = h->per[a];
        A.P[a] = PQ + a * h->N;
        A.Q[a] = PQ + (3 + a) * h->N;
    }
    A.diag = h->diag_ns[set];
    A.scale = P.dth;
}

// U views of a work buffer
double* U_ec(rhi_ctx* h, int b) { return h->U[b]; }
double* U_n(rhi_ctx* h, int b) { return h->U[b] + h->N; }
double* U_E(rhi_ctx* h, int b) { return h->U[b] + (long long)(1 + h->ns) * h->N; }

int validate_params(const rhi_params* p) {
    if (p->n_species != 0 && p->n_species != 1 && p->n_species != 3) return 0;
    if (p->n_species == 1 && p->y_he != 0.0) return 0;
    if ((p->model == RHI_MODEL_LTE) != (p->n_species == 0)) return 0;
    if (p->model == RHI_MODEL_LTE &&
        (!(p->kappa_total >= 0.0) || !(p->kappa_planck >= 0.0) || !(p->mu > 0.0) ||
         p->guess == RHI_GUESS_LEARNED))
        return 0;
    if (!(p->y_he >= 0.0)) return 0;
    if (!(p->theta > 0.0 && p->theta <= 1.0)) return 0;
    if (!(p->u_e > 0.0 && p->u_n > 0.0 && p->u_E > 0.0)) return 0;
    if (!(p->tau > 0.0 && p->tau < 1.0)) return 0;
    if (!(p->lam_min > 0.0 && p->lam_min <= 1.0)) return 0;
    if (!(p->growth_max >= 1.0) || p->watchdog < 0) return 0;
    if (p->max_newton < 0 || p->max_pcg < 1) return 0;
    if (p->guess < 0 || p->guess > RHI_GUESS_LEARNED) return 0;
    if (!(p->mlp_gate >= 0.0) || !(p->mlp_ood >= 0.0) || p->mlp_restart < 0 || p->mlp_retry < 0)
        return 0;
    if (p->precond < 0 || p->precond > RHI_PRECOND_MG_FP32) return 0;
    if (p->mg_levels < 1 || p->mg_pre < 1 || p->mg_post < 0 || p->mg_coarse_sweeps < 1) return 0;
    if (p->limiter_jacobian < 0 || p->limiter_jacobian > 2) return 0;
    if (p->mg_matrix != 0 && p->mg_matrix != 1) return 0;
    if (!(p->krylov_restart < 1.0)) return 0;
    if (p->predict_final != 0 && p->predict_final != 1) return 0;
    if (p->krylov_graph != 0 && p->krylov_graph != 1) return 0;
    if (!(p->mg_omega > 0.0 && p->mg_omega <= 1.0)) return 0;
    if (p->vcycle_graph != 0 && p->vcycle_graph != 1) return 0;
    if (p->dt_norm < -1 || !(p->dt_tau_tol > 0.0)) return 0;
    return 1;
}

// ---- learned guess helpers

enum { SCR_ACT = 0, SCR_DEL, SCR_PART, SCR_X, SCR_Y, SCR_G };

template <typename T>
int scratch(rhi_ctx* h, int slot, size_t count, T** out) {
    rhi_ctx::Scratch& s = h->mlp_scr[slot];
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (s.bytes < bytes) {
        if (s.p) CK(cudaStreamSynchronize(h->st));
        if (s.p) cudaFree(s.p);
        s.p = nullptr;
        s.bytes = 0;
        CK(cudaMalloc(&s.p, bytes));
        s.bytes = bytes;
    }
    *out = (T*)s.p;
    return RHI_OK;
}

MlpArgs mlp_args(const rhi_ctx* h, double dt, double a) {
    MlpArgs A{};
    A.N = h->N;
    A.ns = h->ns;
    A.y_he = h->prm.y_he;
    A.iu_E = 1.0 / h->prm.u_E;
    A.iu_e = 1.0 / h->prm.u_e;
    A.iu_n = 1.0 / h->prm.u_n;
    A.dt = dt;
    A.gam_per_E = C_LIGHT * h->prm.pgam[0] / (a * a * a);
    A.E = h->E_s; A.e = h->e_s; A.n = h->n_s; A.nH = h->nH; A.src = h->src;
    A.gate = (float)h->prm.mlp_gate;
    A.ood = (float)h->prm.mlp_ood;
    A.isothermal = h->prm.isothermal;
    if (h->have_prev) {
        A.E_p = h->E_p; A.e_p = h->e_p; A.n_p = h->n_p;
        A.ldt_ratio = (float)std::log10(dt / h->dt_prev);
    }
    return A;
}

// host copy of the master weights -> BF16 inference copy on the device
int mlp_repack(rhi_ctx* h) {
    std::vector<float> w(RHI_MLP_NWEIGHTS);
    CK(cudaMemcpyAsync(w.data(), h->mlp_w, w.size() * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    MlpPacked pk;
    mlp_pack(w.data(), &pk);
    CK(cudaMemcpyAsync(h->mlp_pk, &pk, sizeof pk, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return RHI_OK;
}

// forward + backward of m samples (device X, Y) into h->mlp_g; squared-error block sums in
// part (ceil(m / block) entries)
int mlp_grad(rhi_ctx* h, const float* X, const float* Y, long long m, double* part) {
    float *act, *del;
    int rc;
    if ((rc = scratch(h, SCR_ACT, (size_t)m * ACT_STRIDE, &act))) return rc;
    if ((rc = scratch(h, SCR_DEL, (size_t)m * DEL_STRIDE, &del))) return rc;
    {
        Scope s(h->prof, "mlp_fwd_bwd");
        CK(launch_mlp_fwd_bwd(h->mlp_w, X, Y, m, act, del, part, h->st));
    }
    {
        Scope s(h->prof, "mlp_wgrad");
        CK(launch_mlp_wgrad(act, del, m, h->mlp_g, h->st));
    }
    return RHI_OK;
}

}  // namespace

// =============================================================================================
// C ABI

extern "C" {

int rhi_params_default(rhi_params* p, int n_species) {
    if (!p || (n_species != 0 && n_species != 1 && n_species != 3)) return RHI_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->n_species = n_species;
    p->y_he = 0.0;
    p->theta = 0.51;
    p->m_grey = 1;
    p->isothermal = 0;
    p->limiter = 1;
    p->kappa_floor = 1e-40;
    p->u_e = p->u_n = p->u_E = 1.0;
    p->tau = 0.99;
    p->lam_min = 1.0 / 16.0;
    p->mlp_gate = 1e-3;
    p->mlp_ood = 6.0;
    p->mlp_restart = 12;
    p->mlp_retry = 4;
    p->growth_max = 1e3;
    p->watchdog = 3;
    p->limiter_jacobian = 0;
    p->max_newton = 50;
    p->max_pcg = 200;
    p->guess = RHI_GUESS_PREVIOUS;
    p->precond = RHI_PRECOND_MG_FP64;
    p->mg_levels = 6;
    p->mg_pre = 2;
    p->mg_post = 2;
    p->mg_coarse_sweeps = 16;
    p->mg_omega = 0.9;
    p->vcycle_graph = 1;
    p->mg_matrix = 1;
    p->krylov_restart = -1.0;
    p->predict_final = 1;
    p->krylov_graph = 1;
    p->dt_norm = 0;
    p->dt_tau_tol = 0.01;
    p->model = n_species == 0 ? RHI_MODEL_LTE : RHI_MODEL_IONIZATION;
    p->kappa_total = 0.0;
    p->kappa_planck = 0.0;
    p->mu = 0.6;
    return rhi_grey_constants(RHI_SPECTRUM_MONO, 13.6 * EV, n_species, p->sk, p->pgam, p->ph,
                              &p->photon_energy);
}

int rhi_create(const rhi_grid* grid, const rhi_bc* bc, const rhi_params* params, void* stream,
               rhi_handle* out) {
    if (!grid || !bc || !params || !out) return RHI_ERR_ARG;
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0.0)) return RHI_ERR_ARG;
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1LL << 31)) return RHI_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        const int lo = bc->kind[2 * a], hi = bc->kind[2 * a + 1];
        if (lo < RHI_BC_ZERO_FLUX || lo > RHI_BC_DIRICHLET || hi < RHI_BC_ZERO_FLUX ||
            hi > RHI_BC_DIRICHLET || (lo == RHI_BC_PERIODIC) != (hi == RHI_BC_PERIODIC))
            return RHI_ERR_ARG;
        for (int s = 0; s < 2; ++s)
            if (bc->kind[2 * a + s] == RHI_BC_DIRICHLET &&
                !(bc->value[2 * a + s] > 0.0 && std::isfinite(bc->value[2 * a + s])))
                return RHI_ERR_ARG;
    }
    if (!validate_params(params)) return RHI_ERR_ARG;

    rhi_ctx* h = new rhi_ctx();
    h->grid = *grid;
    h->bc = *bc;
    h->prm = *params;
    h->ns = params->n_species;
    h->nv = h->ns + 2;
    h->nm = h->ns + 1;
    h->N = N;
    for (int a = 0; a < 3; ++a) h->per[a] = bc->kind[2 * a] == RHI_BC_PERIODIC;
    h->st = (cudaStream_t)stream;
    h->prof.st = h->st;

    int rc = RHI_OK;
    auto A = [&](double** p, size_t n) { if (!rc) rc = dalloc(h, p, n); };
    A(&h->E_s, N); A(&h->e_s, N); A(&h->n_s, (size_t)h->ns * N); A(&h->nH, N); A(&h->src, N);
    A(&h->Tiso, N);
    if (h->ns > 0) { A(&h->E_p, N); A(&h->e_p, N); A(&h->n_p, (size_t)h->ns * N); }
    for (int b = 0; b < 2; ++b) {
        A(&h->U[b], (size_t)h->nv * N); A(&h->kap[b], N); A(&h->W[b], 3 * (size_t)N);
        A(&h->diag[b], N); A(&h->rhs[b], N); A(&h->fMt[b], (size_t)h->nm * N);
        A(&h->MiU[b], (size_t)h->nm * N);
        if (params->limiter_jacobian) { A(&h->PQ[b], 6 * (size_t)N); A(&h->diag_ns[b], N); }
        if (params->limiter_jacobian == 2) A(&h->Kf[b], 3 * (size_t)N);
    }
    if (params->limiter_jacobian) {
        A(&h->rh, N); A(&h->v, N); A(&h->s, N); A(&h->t, N); A(&h->ph, N); A(&h->sh, N);
    }
    A(&h->g, (size_t)h->nv * N);
    if (params->dt_norm) A(&h->Upred, (size_t)h->nv * N);
    A(&h->x, N); A(&h->r, N); A(&h->z, N); A(&h->p, N); A(&h->q, N);
    const long long nparts = std::max<long long>((N + cell_block_size() - 1) / cell_block_size(),
                                                 2 * (long long)stream_blocks(N));
    A(&h->partials, (size_t)nparts);
    A(&h->scal, S_NSCAL);
    if (!rc) rc = dalloc(h, &h->d_flag, 1);
    if (!rc) rc = dalloc(h, &h->table, (size_t)NBINS * NRATES);
    if (!rc) rc = mg_build_levels(h);
    if (!rc) {
        cudaError_t e = cudaMallocHost(&h->h_scal, sizeof(double) * S_NSCAL);
        if (e == cudaSuccess) e = cudaMallocHost(&h->h_ctl, sizeof(double) * 3);
        if (e == cudaSuccess) e = cudaMallocHost(&h->h_kerr, sizeof(int));
        if (e != cudaSuccess) rc = fail(h, RHI_ERR_CUDA, "cudaMallocHost");
        if (!rc) {
            *h->h_kerr = 0;
            e = linear_kernels_init();
            if (e != cudaSuccess) rc = fail(h, RHI_ERR_CUDA, std::string("multigrid kernels: ") + cudaGetErrorString(e));
        }
    }
    if (!rc) {
        std::vector<double2> tab = build_rate_table();
        cudaError_t e = cudaMemcpy(h->table, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(h->src, 0, N * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(h->scal, 0, S_NSCAL * sizeof(double));
        if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
        if (e != cudaSuccess) rc = fail(h, RHI_ERR_CUDA, std::string("rhi_create: ") + cudaGetErrorString(e));
    }
    if (rc) {
        rhi_destroy(h);
        return rc;
    }
    *out = h;
    return RHI_OK;
}

void rhi_destroy(rhi_handle h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    if (h->h_kerr) cudaFreeHost(h->h_kerr);
    if (h->kst) cudaStreamSynchronize(h->kst);
    for (auto& c : h->kg) if (c.exec) cudaGraphExecDestroy(c.exec);
    if (h->kst) cudaStreamDestroy(h->kst);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->vg.st) cudaStreamSynchronize(h->vg.st);
    if (h->vg.exec) cudaGraphExecDestroy(h->vg.exec);
    if (h->vg.ev0) cudaEventDestroy(h->vg.ev0);
    if (h->vg.ev1) cudaEventDestroy(h->vg.ev1);
    if (h->vg.st) cudaStreamDestroy(h->vg.st);
    delete h;
}

const char* rhi_last_error(rhi_handle h) { return h ? h->err.c_str() : "null handle"; }

const char* rhi_status_string(int s) {
    switch (s) {
        case RHI_OK: return "ok";
        case RHI_ERR_ARG: return "invalid argument";
        case RHI_ERR_CUDA: return "CUDA error";
        case RHI_ERR_NONCONVERGED: return "Newton iteration did not converge";
        case RHI_ERR_NONPHYSICAL: return "non-physical state or CG breakdown";
        case RHI_ERR_STATE: return "no state set";
        default: return "unknown status";
    }
}

int rhi_set_state(rhi_handle h, const double* E, const double* e, const double* n,
                  const double* n_H, const double* src, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (!E || !e || (!n && h->ns > 0) || !n_H) return fail(h, RHI_ERR_ARG, "rhi_set_state: null field");
    const long long N = h->N;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(h->E_s, E, N * sizeof(double), kind, h->st));
    CK(cudaMemcpyAsync(h->e_s, e, N * sizeof(double), kind, h->st));
    if (h->ns > 0) CK(cudaMemcpyAsync(h->n_s, n, (size_t)h->ns * N * sizeof(double), kind, h->st));
    CK(cudaMemcpyAsync(h->nH, n_H, N * sizeof(double), kind, h->st));
    if (src) CK(cudaMemcpyAsync(h->src, src, N * sizeof(double), kind, h->st));
    else CK(cudaMemsetAsync(h->src, 0, N * sizeof(double), h->st));
    StepParams P = make_params(h, 1.0, 1.0, 0.0);
    CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->st));
    {
        Scope s(h->prof, "check_state");
        CK(launch_check_state(P, h->ns, h->E_s, h->e_s, h->n_s, h->nH, h->d_flag, h->st));
    }
    if (h->prm.isothermal) {
        Scope s(h->prof, "temperature");
        CK(launch_temperature(P, h->ns, h->e_s, h->n_s, h->nH, h->Tiso, h->st));
    }
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    h->have_linear = false;
    if (bad) {
        h->have_state = false;
        return fail(h, RHI_ERR_NONPHYSICAL, "rhi_set_state: need E > 0, e > 0, n_H > 0, species >= 0, finite");
    }
    h->have_state = true;
    return RHI_OK;
}

int rhi_set_sources(rhi_handle h, int nsrc, const int* ijk, const double* rate) {
    if (!h) return RHI_ERR_ARG;
    if (nsrc < 0 || (nsrc > 0 && (!ijk || !rate))) return fail(h, RHI_ERR_ARG, "rhi_set_sources: bad arguments");
    const double vol = h->grid.dx * h->grid.dx * h->grid.dx;
    for (int s = 0; s < nsrc; ++s) {
        const int i = ijk[3 * s], j = ijk[3 * s + 1], k = ijk[3 * s + 2];
        if (i < 0 || j < 0 || k < 0 || i >= h->grid.nx || j >= h->grid.ny || k >= h->grid.nz)
            return fail(h, RHI_ERR_ARG, "rhi_set_sources: source outside the grid");
        if (!(rate[s] >= 0.0)) return fail(h, RHI_ERR_ARG, "rhi_set_sources: negative rate");
    }
    for (int s = 0; s < nsrc; ++s) {
        const long long c = ijk[3 * s] + (long long)h->grid.nx * (ijk[3 * s + 1] + (long long)h->grid.ny * ijk[3 * s + 2]);
        Scope sc(h->prof, "deposit_source");
        CK(launch_deposit(c, rate[s] * h->prm.photon_energy / vol, h->src, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return RHI_OK;
}

int rhi_get_state(rhi_handle h, double* E, double* e, double* n, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_get_state: no state");
    const long long N = h->N;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (E) CK(cudaMemcpyAsync(E, h->E_s, N * sizeof(double), kind, h->st));
    if (e) CK(cudaMemcpyAsync(e, h->e_s, N * sizeof(double), kind, h->st));
    if (n) CK(cudaMemcpyAsync(n, h->n_s, (size_t)h->ns * N * sizeof(double), kind, h->st));
    CK(cudaStreamSynchronize(h->st));
    return RHI_OK;
}

int rhi_get_stats(rhi_handle h, rhi_stats* out) {
    if (!h || !out) return RHI_ERR_ARG;
    *out = h->stats;
    return RHI_OK;
}

int rhi_set_profiling(rhi_handle h, int on) {
    if (!h) return RHI_ERR_ARG;
    h->prof.on = on != 0;
    h->prof.acc.clear();
    return RHI_OK;
}

int rhi_set_profiling_names(rhi_handle h, const char* names) {
    if (!h) return RHI_ERR_ARG;
    h->prof.only.clear();
    if (names) {
        std::string s(names);
        size_t a = 0;
        while (a <= s.size()) {
            size_t b = s.find(',', a);
            if (b == std::string::npos) b = s.size();
            if (b > a) h->prof.only.push_back(s.substr(a, b - a));
            a = b + 1;
        }
    }
    return RHI_OK;
}

int rhi_kernel_times(rhi_handle h, int max, char* names, double* total_ms, int* launches) {
    if (!h) return -RHI_ERR_ARG;
    h->prof.resolve();
    int i = 0;
    for (auto& kv : h->prof.acc) {
        if (i < max) {
            if (names) {
                std::strncpy(names + 48 * i, kv.first.c_str(), 47);
                names[48 * i + 47] = 0;
            }
            if (total_ms) total_ms[i] = kv.second.first;
            if (launches) launches[i] = kv.second.second;
        }
        ++i;
    }
    return i;
}

int rhi_linearize(rhi_handle h, double dt, double a, double adot, double* f, double* S_diag,
                  double* S_lo, double* S_hi, double* rhs, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_linearize: no state");
    if (!(dt > 0.0) || !(a > 0.0)) return fail(h, RHI_ERR_ARG, "rhi_linearize: dt > 0 and a > 0 required");
    const StepParams P = make_params(h, dt, a, adot);
    int rc;
    if ((rc = kappa(h, P, h->n_s, h->kap[0]))) return rc;
    if ((rc = faces(h, P, h->E_s, h->kap[0], 0))) return rc;
    PhysBuffers B = state_buffers(h);
    B.W = h->W[0];
    B.PQ = h->PQ[0]; B.diag_ns = h->diag_ns[0];
    B.diag = h->diag[0]; B.rhs = h->rhs[0]; B.fMt = h->fMt[0]; B.MiU = h->MiU[0];
    // the residual goes straight to a device destination, or via a free work buffer
    if (f) B.f_out = on_device ? f : h->U[1];
    if ((rc = cell(h, P, MODE_PREP, B))) return rc;
    if ((rc = schur_kappa(h, P, 0, 0))) return rc;
    set_op0(h, P, 0, h->W[0]);
    if (h->prm.limiter_jacobian) set_opns(h, P, 0, h->PQ[0]);
    if ((rc = precond_setup_newton(h))) return rc;
    const long long N = h->N;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (f && !on_device) CK(cudaMemcpyAsync(f, h->U[1], (size_t)h->nv * N * sizeof(double), kind, h->st));
    const double* dsrc = h->prm.limiter_jacobian ? h->diag_ns[0] : h->diag[0];
    if (S_diag) CK(cudaMemcpyAsync(S_diag, dsrc, N * sizeof(double), kind, h->st));
    if (rhs) CK(cudaMemcpyAsync(rhs, h->rhs[0], N * sizeof(double), kind, h->st));
    if (S_lo || S_hi) {
        // face entries of the Newton matrix (an inspection path: a temporary buffer)
        double* tmp = nullptr;
        CK(cudaMalloc(&tmp, 6 * N * sizeof(double)));
        cudaError_t e = cudaSuccess;
        {
            Scope s(h->prof, "export_faces");
            e = launch_export_faces(P, h->W[0], h->PQ[0], tmp, tmp + 3 * N, h->st);
        }
        if (e == cudaSuccess && S_lo) e = cudaMemcpyAsync(S_lo, tmp, 3 * N * sizeof(double), kind, h->st);
        if (e == cudaSuccess && S_hi) e = cudaMemcpyAsync(S_hi, tmp + 3 * N, 3 * N * sizeof(double), kind, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        cudaFree(tmp);
        if (e != cudaSuccess) return fail(h, RHI_ERR_CUDA, std::string("rhi_linearize: ") + cudaGetErrorString(e));
    }
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    h->have_linear = true;
    return RHI_OK;
}

int rhi_residual(rhi_handle h, double dt, double a, double adot, const double* U, double* f,
                 double* norm, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_residual: no state");
    if (!U || !(dt > 0.0) || !(a > 0.0)) return fail(h, RHI_ERR_ARG, "rhi_residual: bad arguments");
    h->have_linear = false;
    const StepParams P = make_params(h, dt, a, adot);
    const long long N = h->N;
    const size_t bytes = (size_t)h->nv * N * sizeof(double);
    int rc;
    // g^n from the state, then f at the given iterate (work iterate 1, Schur set 1)
    if ((rc = kappa(h, P, h->n_s, h->kap[0]))) return rc;
    if ((rc = faces(h, P, h->E_s, h->kap[0], 0))) return rc;
    PhysBuffers B = state_buffers(h);
    B.W = h->W[0]; B.PQ = h->PQ[0]; B.diag_ns = h->diag_ns[0];
    B.diag = h->diag[0]; B.rhs = h->rhs[0]; B.fMt = h->fMt[0]; B.MiU = h->MiU[0];
    if ((rc = cell(h, P, MODE_PREP, B))) return rc;
    CK(cudaMemcpyAsync(h->U[1], U, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    if ((rc = kappa(h, P, U_n(h, 1), h->kap[1]))) return rc;
    if ((rc = faces(h, P, U_E(h, 1), h->kap[1], 1))) return rc;
    PhysBuffers C = state_buffers(h);
    C.ec = U_ec(h, 1); C.n = U_n(h, 1); C.E = U_E(h, 1); C.W = h->W[1];
    C.PQ = h->PQ[1]; C.diag_ns = h->diag_ns[1];
    C.diag = h->diag[1]; C.rhs = h->rhs[1]; C.fMt = h->fMt[1]; C.MiU = h->MiU[1];
    if (f) C.f_out = on_device ? f : h->U[0];
    if ((rc = cell(h, P, MODE_ITER, C))) return rc;
    double r = 0.0;
    if ((rc = residual_norm(h, ncell_blocks(h), &r))) return rc;
    if (norm) *norm = r;
    if (f && !on_device) CK(cudaMemcpyAsync(f, h->U[0], bytes, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return RHI_OK;
}

int rhi_mlp_guess(rhi_handle h, double dt, double a, double* U0, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (h->ns == 0) return fail(h, RHI_ERR_ARG, "rhi_mlp_guess: the learned guess needs the ionization model");
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_mlp_guess: no state");
    if (!h->mlp_ready) return fail(h, RHI_ERR_STATE, "rhi_mlp_guess: no weights set");
    if (!U0 || !(dt > 0.0) || !(a > 0.0)) return fail(h, RHI_ERR_ARG, "rhi_mlp_guess: bad arguments");
    MlpArgs A = mlp_args(h, dt, a);
    A.U0 = on_device ? U0 : h->U[1];
    {
        Scope s(h->prof, "mlp_guess");
        CK(launch_mlp_infer(A, h->mlp_pk, nullptr, nullptr, 0, 1, h->st));
    }
    if (!on_device)
        CK(cudaMemcpyAsync(U0, h->U[1], (size_t)h->nv * h->N * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->have_linear = false;
    h->prof.resolve();
    return RHI_OK;
}

// after the stream work of a call is done: a staged multigrid sweep that gave up waiting on
// its copies makes the call fail (the flag is cleared for the next call)
int bulk_wait_check(rhi_ctx* h) {
    if (!*h->h_kerr) return RHI_OK;
    *h->h_kerr = 0;
    CK(bulk_wait_flag_clear(h->st));
    CK(cudaStreamSynchronize(h->st));
    return fail(h, RHI_ERR_CUDA, "multigrid: a staged sweep timed out waiting for its copies");
}

int rhi_precond_apply(rhi_handle h, const double* r, double* z, int on_device) {
    if (!h || !r || !z) return RHI_ERR_ARG;
    if (!h->have_linear) return fail(h, RHI_ERR_STATE, "rhi_precond_apply: call rhi_linearize first");
    const long long N = h->N;
    CK(cudaMemcpyAsync(h->q, r, N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    double* zr = nullptr;
    int np = 0;
    int rc = precond_apply(h, h->q, &zr, np);
    if (rc) return rc;
    CK(cudaMemcpyAsync(z, zr, N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(bulk_wait_flag_read(h->h_kerr, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return bulk_wait_check(h);
}

int rhi_implicit_step(rhi_handle h, double dt, double a, double adot, double newton_tol,
                      double lin_tol) {
    if (!h) return RHI_ERR_ARG;
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_implicit_step: no state");
    if (h->prm.guess == RHI_GUESS_LEARNED && !h->mlp_ready)
        return fail(h, RHI_ERR_STATE, "rhi_implicit_step: learned guess without weights");
    if (!(dt > 0.0) || !(a > 0.0) || !(newton_tol > 0.0) || !(lin_tol > 0.0) || !std::isfinite(adot))
        return fail(h, RHI_ERR_ARG, "rhi_implicit_step: need dt > 0, a > 0, tolerances > 0");
    h->have_linear = false;
    rhi_stats& S = h->stats;
    S = rhi_stats{};
    S.status = RHI_OK;
    h->host_syncs = 0;
    const int launches0 = h->prof.launches;
    const StepParams P = make_params(h, dt, a, adot);
    const long long N = h->N;
    const int ns = h->ns;
    LinLaunch L(h->st, &h->prof);
    CK(cudaEventRecord(h->ev0, h->st));
    int rc;

    // ---- g^n and the initial iterate U_0
    if ((rc = kappa(h, P, h->n_s, h->kap[0]))) return rc;
    if ((rc = faces(h, P, h->E_s, h->kap[0], 0))) return rc;
    PhysBuffers B = state_buffers(h);
    B.W = h->W[0];
    B.PQ = h->PQ[0]; B.diag_ns = h->diag_ns[0];
    int cur = -1;            // -1: U_k is the state U^n (e_c = 0); 0 / 1: work buffer
    int set = 0;             // Schur set of U_k
    double res = 0.0;
    S.guess_used = h->prm.guess;
    if (h->prm.guess == RHI_GUESS_PREVIOUS || h->prm.guess == RHI_GUESS_LEARNED) {
        B.diag = h->diag[0]; B.rhs = h->rhs[0]; B.fMt = h->fMt[0]; B.MiU = h->MiU[0];
        B.U0 = h->Upred;                    // the explicit predictor, for the error estimate
        if ((rc = cell(h, P, MODE_PREP, B))) return rc;
        B.U0 = nullptr;
        if ((rc = residual_norm(h, ncell_blocks(h), &res))) return rc;
        if (h->prm.guess == RHI_GUESS_LEARNED && h->mlp_skip > 0) {
            h->mlp_skip -= 1;
            S.guess_used = RHI_GUESS_PREVIOUS;
        } else if (h->prm.guess == RHI_GUESS_LEARNED) {
            // the network's guess into work iterate 1 with its own Schur set; Newton starts
            // from whichever of U^n and the guess has the smaller ||f||
            MlpArgs A = mlp_args(h, dt, a);
            A.U0 = h->U[1];
            {
                Scope s(h->prof, "mlp_guess");
                CK(launch_mlp_infer(A, h->mlp_pk, nullptr, nullptr, 0, 1, h->st));
            }
            if ((rc = kappa(h, P, U_n(h, 1), h->kap[1]))) return rc;
            if ((rc = faces(h, P, U_E(h, 1), h->kap[1], 1))) return rc;
            PhysBuffers C = state_buffers(h);
            C.ec = U_ec(h, 1); C.n = U_n(h, 1); C.E = U_E(h, 1); C.W = h->W[1];
            C.PQ = h->PQ[1]; C.diag_ns = h->diag_ns[1];
            C.diag = h->diag[1]; C.rhs = h->rhs[1]; C.fMt = h->fMt[1]; C.MiU = h->MiU[1];
            if ((rc = cell(h, P, MODE_ITER, C))) return rc;
            double rg = 0.0;
            if ((rc = residual_norm(h, ncell_blocks(h), &rg))) return rc;
            S.res_guess_prev = res;
            if (rg < res) {
                cur = 1;
                set = 1;
                res = rg;
            } else {
                S.guess_used = RHI_GUESS_PREVIOUS;
                h->mlp_skip = h->prm.mlp_retry;
            }
        }
    } else {
        B.U0 = h->U[0];
        if ((rc = cell(h, P, MODE_PREP_PREDICT, B))) return rc;
        if (h->Upred)
            CK(cudaMemcpyAsync(h->Upred, h->U[0], (size_t)h->nv * N * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->st));
        cur = 0;
        if ((rc = kappa(h, P, U_n(h, 0), h->kap[0]))) return rc;
        if ((rc = faces(h, P, U_E(h, 0), h->kap[0], 0))) return rc;
        PhysBuffers C = state_buffers(h);
        C.ec = U_ec(h, 0); C.n = U_n(h, 0); C.E = U_E(h, 0); C.W = h->W[0];
        C.PQ = h->PQ[0]; C.diag_ns = h->diag_ns[0];
        C.diag = h->diag[0]; C.rhs = h->rhs[0]; C.fMt = h->fMt[0]; C.MiU = h->MiU[0];
        if ((rc = cell(h, P, MODE_ITER, C))) return rc;
        if ((rc = residual_norm(h, ncell_blocks(h), &res))) return rc;
    }
    S.res_initial = res;
    if (!std::isfinite(res)) { S.status = RHI_ERR_NONPHYSICAL; return fail(h, RHI_ERR_NONPHYSICAL, "non-finite initial residual"); }

    // ---- Newton iteration
    int k = 0;
    double r_best = res;
    int bad = 0;
    S.res_history[0] = res;
    int k_start = 0;         // iteration at which the current start was taken
    double res_prev = 0.0;   // ||f|| of the iterate before U_k (0: none since the start)
    while (!(res < newton_tol) && k < h->prm.max_newton) {
        const bool stalled = k - k_start >= 2 && k < RHI_MAX_HISTORY &&
                             res > 0.9 * S.res_history[k - 2];
        if (S.guess_used == RHI_GUESS_LEARNED && h->prm.mlp_restart > 0 &&
            (k - k_start >= h->prm.mlp_restart || stalled)) {
            // the learned start has not converged in mlp_restart iterations: restart from U^n
            if ((rc = kappa(h, P, h->n_s, h->kap[0]))) return rc;
            if ((rc = faces(h, P, h->E_s, h->kap[0], 0))) return rc;
            PhysBuffers C = state_buffers(h);
            C.W = h->W[0]; C.PQ = h->PQ[0]; C.diag_ns = h->diag_ns[0];
            C.diag = h->diag[0]; C.rhs = h->rhs[0]; C.fMt = h->fMt[0]; C.MiU = h->MiU[0];
            if ((rc = cell(h, P, MODE_PREP, C))) return rc;
            if ((rc = residual_norm(h, ncell_blocks(h), &res))) return rc;
            cur = -1;
            set = 0;
            r_best = res;
            bad = 0;
            k_start = k;
            res_prev = 0.0;
            S.guess_used = RHI_GUESS_PREVIOUS;
            S.guess_restarts = 1;
            if (res < newton_tol) break;
        }
        const double* Wk = h->W[cur < 0 ? 0 : cur];
        if ((rc = schur_kappa(h, P, cur < 0 ? 0 : cur, set))) return rc;
        set_op0(h, P, set, Wk);
        if (h->prm.limiter_jacobian) set_opns(h, P, set, h->PQ[cur < 0 ? 0 : cur]);
        if ((rc = precond_setup_newton(h))) return rc;
        int its = 0;
        // BiCGStab broke down (where free streaming makes the advective part of the matrix
        // dominate): this Newton iteration takes the direction of the symmetric lagged-D
        // matrix instead, solved by CG with that matrix's V-cycle
        auto krylov_fallback = [&]() -> int {
            S.krylov_fallbacks += 1;
            S.pcg_its += its;
            int r2;
            if (h->pc_nonsym && (r2 = precond_setup(h, h->op0, false))) return r2;
            return pcg(h, h->rhs[set], lin_tol * res, &its);
        };
        bool deferred = false;
        if (h->prm.limiter_jacobian) {
            rc = bicgstab(h, h->rhs[set], lin_tol * res, &its, true);
            deferred = rc == RHI_OK && its < 0;
            if (rc == RHI_ERR_NONPHYSICAL) rc = krylov_fallback();
            if (rc) { S.status = rc; return rc; }
        } else if ((rc = pcg(h, h->rhs[set], lin_tol * res, &its))) {
            S.status = rc;
            return rc;
        }
        const int t = (cur == 0) ? 1 : 0;
        const double* ec0 = cur < 0 ? nullptr : U_ec(h, cur);
        const double* n0 = cur < 0 ? h->n_s : U_n(h, cur);
        const double* E0 = cur < 0 ? h->E_s : U_E(h, cur);
        // the trial iterate's faces, residual and (unless resid_only) Schur set
        auto evaluate = [&](double* rt, bool resid_only) -> int {
            int r2;
            if (resid_only) {
                if ((r2 = faces_w(h, P, U_E(h, t), h->kap[t], t))) return r2;
            } else if ((r2 = faces(h, P, U_E(h, t), h->kap[t], t))) {
                return r2;
            }
            PhysBuffers C = state_buffers(h);
            C.ec = U_ec(h, t); C.n = U_n(h, t); C.E = U_E(h, t); C.W = h->W[t];
            C.PQ = h->PQ[t]; C.diag_ns = h->diag_ns[1 - set];
            C.diag = h->diag[1 - set]; C.rhs = h->rhs[1 - set];
            C.fMt = h->fMt[1 - set]; C.MiU = h->MiU[1 - set];
            if ((r2 = cell(h, P, resid_only ? MODE_RESID : MODE_ITER, C))) return r2;
            return residual_norm(h, ncell_blocks(h), rt);
        };
        // U_k + min(lam, cap) S_k into buffer t, then its evaluation
        auto trial = [&](double lam, double* rt, bool resid_only = false) -> int {
            {
                Scope s(h->prof, "update_recover_limit");
                CK(launch_update(P, ns, lam, ec0, n0, E0, h->e_s, h->nH, h->x, h->fMt[set],
                                 h->MiU[set], U_ec(h, t), U_n(h, t), U_E(h, t), h->kap[t], h->st));
            }
            return evaluate(rt, resid_only);
        };
        // The full step is expected to end the iteration when the quadratic model through the
        // last two residuals, ||f_k+1|| ~ ||f_k||^2 ||f_k|| / ||f_k-1||^2, puts it below a tenth
        // of the tolerance: its iterate is then evaluated for f alone, and again in full only
        // if it did not converge (the Jacobian and Schur system of the last iterate are not
        // needed).
        bool resid_only = false;
        if (h->prm.predict_final && k - k_start >= 1 && res_prev > 0.0) {
            const double q = res / res_prev;
            resid_only = q * q * res < 0.1 * newton_tol;
        }
        // watchdog line search (Sec. 3.2, item 2): full steps, non-monotone for at most
        // `watchdog` iterations without a new best ||f||, else Armijo backtracking
        double rt = 0.0;
        if ((rc = trial(1.0, &rt, resid_only))) return rc;
        if (deferred) {
            // the full step's residual read also brought the Krylov solve's outcome back
            rc = bicg_outcome(h, &its);
            if (rc == RHI_ERR_NONPHYSICAL) {
                if ((rc = krylov_fallback())) { S.status = rc; return rc; }
                if ((rc = trial(1.0, &rt))) return rc;        // in full
                resid_only = false;
            } else if (rc) {
                S.status = rc;
                return rc;
            }
        }
        if (resid_only) {
            S.final_predicted += 1;
            if (!(rt < newton_tol)) {
                // not converged after all: the same iterate in full (its residual again, the
                // Jacobian and the Schur system for the next Newton iteration)
                S.final_missed += 1;
                if ((rc = evaluate(&rt, false))) return rc;
            }
        }
        S.pcg_its += its;
        if (rt <= (1.0 - 1e-4) * r_best) {
            r_best = rt;
            bad = 0;
        } else if (bad < h->prm.watchdog && rt <= h->prm.growth_max * r_best) {
            bad += 1;
        } else {
            double lam = 1.0;
            while (!(rt <= (1.0 - 1e-4 * lam) * res)) {
                if (lam * 0.5 < h->prm.lam_min) { S.lam_min_steps += 1; break; }
                lam *= 0.5;
                S.backtracks += 1;
                if ((rc = trial(lam, &rt))) return rc;
            }
            bad = 0;
            r_best = std::min(r_best, rt);
        }
        cur = t;
        set = 1 - set;
        res_prev = res;
        res = rt;
        ++k;
        if (k < RHI_MAX_HISTORY) S.res_history[k] = res;
        if (!std::isfinite(res)) break;
    }
    S.newton_its = k;
    S.res_final = res;
    if (!std::isfinite(res)) {
        S.status = RHI_ERR_NONPHYSICAL;
        S.launches = h->prof.launches - launches0;
        h->prof.resolve();
        return fail(h, RHI_ERR_NONPHYSICAL, "non-finite residual during Newton");
    }
    if (!(res < newton_tol)) {
        S.status = RHI_ERR_NONCONVERGED;
        S.launches = h->prof.launches - launches0;
        h->prof.resolve();
        char buf[160];
        std::snprintf(buf, sizeof buf, "Newton: ||f|| = %.3e >= %.3e after %d iterations", res, newton_tol, k);
        return fail(h, RHI_ERR_NONCONVERGED, buf);
    }
    // ---- error estimate against the explicit predictor (Sec. 3.2.3)
    if (h->prm.dt_norm) {
        const int nb = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
        const double pn = h->prm.dt_norm < 0 ? -1.0 : (double)h->prm.dt_norm;
        {
            Scope s(h->prof, "time_error");
            CK(launch_time_error(P, ns, cur < 0 ? nullptr : U_ec(h, cur), cur < 0 ? h->n_s : U_n(h, cur),
                                 cur < 0 ? h->E_s : U_E(h, cur), h->Upred, pn, h->partials, nb, h->st));
        }
        LinLaunch Le(h->st, &h->prof);
        CK(Le.reduce(h->partials, nb, h->scal, pn < 0.0 ? RED_MAX : RED_SUM, S_TMP));
        double v = 0.0;
        if ((rc = read_scalar(h, S_TMP, &v))) return rc;
        S.eps_loc = pn < 0.0 ? v : std::pow(v / ((double)N * h->nv), 1.0 / pn);
        S.dt_next = S.eps_loc > 0.0 ? h->prm.dt_tau_tol * dt / S.eps_loc : HUGE_VAL;
    }
    // ---- accept: U^n -> the previous state (the learned guess's features), U^{n+1} -> state,
    // e^{n+1} = e_h + e_c
    if (h->E_p) {
        CK(cudaMemcpyAsync(h->E_p, h->E_s, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(h->e_p, h->e_s, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(h->n_p, h->n_s, (size_t)ns * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        h->have_prev = true;
        h->dt_prev = dt;
    }
    if (cur >= 0) {
        {
            Scope s(h->prof, "finalize_energy");
            CK(launch_finalize(P, ns, U_ec(h, cur), h->e_s, h->st));
        }
        CK(cudaMemcpyAsync(h->n_s, U_n(h, cur), (size_t)ns * N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(h->E_s, U_E(h, cur), N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    }
    CK(bulk_wait_flag_read(h->h_kerr, h->st));
    CK(cudaEventRecord(h->ev1, h->st));
    CK(cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    S.ms = ms;
    S.launches = h->prof.launches - launches0;
    S.host_syncs = h->host_syncs + 1;          // and the final event wait
    h->prof.resolve();
    if ((rc = bulk_wait_check(h))) { S.status = rc; return rc; }
    return RHI_OK;
}

int rhi_advance(rhi_handle h, double t_end, double dt0, double dt_min, double dt_max, double a,
                double adot, double newton_tol, double lin_tol, int max_steps, double* t_reached,
                int* steps) {
    if (!h) return RHI_ERR_ARG;
    if (!h->prm.dt_norm) return fail(h, RHI_ERR_ARG, "rhi_advance: params.dt_norm is 0");
    if (!(t_end >= 0.0) || !(dt0 > 0.0) || !(dt_min >= 0.0) || !(dt_max >= dt_min) || max_steps < 0)
        return fail(h, RHI_ERR_ARG, "rhi_advance: bad arguments");
    double t = 0.0, dt = std::min(dt0, dt_max);
    int n = 0, rc = RHI_OK;
    while (t < t_end * (1.0 - 1e-12) && n < max_steps) {
        double d = std::min(dt, t_end - t);
        rc = rhi_implicit_step(h, d, a, adot, newton_tol, lin_tol);
        while ((rc == RHI_ERR_NONCONVERGED || rc == RHI_ERR_NONPHYSICAL) && 0.5 * d >= dt_min &&
               0.5 * d > 0.0) {
            d *= 0.5;                           // the state is unchanged by a failed step
            rc = rhi_implicit_step(h, d, a, adot, newton_tol, lin_tol);
        }
        if (rc) break;
        t += d;
        ++n;
        dt = std::min(std::max(h->stats.dt_next, dt_min), dt_max);
    }
    if (t_reached) *t_reached = t;
    if (steps) *steps = n;
    if (rc) return rc;
    if (t < t_end * (1.0 - 1e-12))
        return fail(h, RHI_ERR_NONCONVERGED, "rhi_advance: max_steps reached before t_end");
    return RHI_OK;
}

// ---- learned guess (an addition to the paper's method)

int rhi_mlp_set_weights(rhi_handle h, const float* w, size_t n) {
    if (!h) return RHI_ERR_ARG;
    if (!w || n != (size_t)RHI_MLP_NWEIGHTS)
        return fail(h, RHI_ERR_ARG, "rhi_mlp_set_weights: need RHI_MLP_NWEIGHTS weights");
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(w[q])) return fail(h, RHI_ERR_ARG, "rhi_mlp_set_weights: non-finite weight");
    for (int q = 0; q < RHI_MLP_IN; ++q)
        if (!(w[n - RHI_MLP_IN + q] > 0.0f)) return fail(h, RHI_ERR_ARG, "rhi_mlp_set_weights: scale must be > 0");
    int rc = RHI_OK;
    if (!h->mlp_w) {
        if (!rc) rc = dalloc(h, &h->mlp_w, n);
        if (!rc) rc = dalloc(h, &h->mlp_m1, n);
        if (!rc) rc = dalloc(h, &h->mlp_m2, n);
        if (!rc) rc = dalloc(h, &h->mlp_g, n);
        if (!rc) rc = dalloc(h, &h->mlp_pk, 1);
        if (rc) return rc;
    }
    CK(cudaMemcpyAsync(h->mlp_w, w, n * sizeof(float), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemsetAsync(h->mlp_m1, 0, n * sizeof(float), h->st));
    CK(cudaMemsetAsync(h->mlp_m2, 0, n * sizeof(float), h->st));
    CK(cudaMemsetAsync(h->mlp_g, 0, n * sizeof(float), h->st));
    h->mlp_t = 0;
    h->mlp_skip = 0;
    if ((rc = mlp_repack(h))) return rc;
    h->mlp_ready = true;
    return RHI_OK;
}

int rhi_mlp_get_weights(rhi_handle h, float* w, size_t n) {
    if (!h) return RHI_ERR_ARG;
    if (!h->mlp_ready) return fail(h, RHI_ERR_STATE, "rhi_mlp_get_weights: no weights set");
    if (!w || n != (size_t)RHI_MLP_NWEIGHTS)
        return fail(h, RHI_ERR_ARG, "rhi_mlp_get_weights: need RHI_MLP_NWEIGHTS weights");
    CK(cudaMemcpyAsync(w, h->mlp_w, n * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return RHI_OK;
}

int rhi_mlp_features(rhi_handle h, double dt, double a, float* X, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (h->ns == 0) return fail(h, RHI_ERR_ARG, "rhi_mlp_features: the learned guess needs the ionization model");
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_mlp_features: no state");
    if (!X || !(dt > 0.0) || !(a > 0.0)) return fail(h, RHI_ERR_ARG, "rhi_mlp_features: bad arguments");
    const MlpArgs A = mlp_args(h, dt, a);
    float* dst = X;
    int rc;
    if (!on_device && (rc = scratch(h, SCR_X, (size_t)h->N * MLP_IN, &dst))) return rc;
    {
        Scope s(h->prof, "mlp_features");
        CK(launch_mlp_features(A, dst, h->st));
    }
    if (!on_device)
        CK(cudaMemcpyAsync(X, dst, (size_t)h->N * MLP_IN * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return RHI_OK;
}

int rhi_mlp_targets(rhi_handle h, const double* E_old, const double* e_old, const double* n_old,
                    float* Y, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (h->ns == 0) return fail(h, RHI_ERR_ARG, "rhi_mlp_targets: the learned guess needs the ionization model");
    if (!h->have_state) return fail(h, RHI_ERR_STATE, "rhi_mlp_targets: no state");
    if (!E_old || !e_old || !n_old || !Y) return fail(h, RHI_ERR_ARG, "rhi_mlp_targets: null argument");
    const long long N = h->N;
    const double *E0 = E_old, *e0 = e_old, *n0 = n_old;
    float* dst = Y;
    int rc;
    if (!on_device) {
        // the old state goes through the second work iterate (E | e | n), nv * N doubles
        double* b = h->U[1];
        CK(cudaMemcpyAsync(b, E_old, N * sizeof(double), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(b + N, e_old, N * sizeof(double), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(b + 2 * N, n_old, (size_t)h->ns * N * sizeof(double), cudaMemcpyHostToDevice, h->st));
        E0 = b; e0 = b + N; n0 = b + 2 * N;
        if ((rc = scratch(h, SCR_Y, (size_t)N * MLP_OUT, &dst))) return rc;
        h->have_linear = false;
    }
    const MlpArgs A = mlp_args(h, 1.0, 1.0);
    {
        Scope s(h->prof, "mlp_targets");
        CK(launch_mlp_targets(A, E0, e0, n0, dst, h->st));
    }
    if (!on_device)
        CK(cudaMemcpyAsync(Y, dst, (size_t)N * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return RHI_OK;
}

int rhi_mlp_forward(rhi_handle h, const float* X, float* Y, long long n, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (!h->mlp_ready) return fail(h, RHI_ERR_STATE, "rhi_mlp_forward: no weights set");
    if (!X || !Y || n < 0) return fail(h, RHI_ERR_ARG, "rhi_mlp_forward: bad arguments");
    if (n == 0) return RHI_OK;
    const float* src = X;
    float* dst = Y;
    int rc;
    if (!on_device) {
        float *xs, *ys;
        if ((rc = scratch(h, SCR_X, (size_t)n * MLP_IN, &xs))) return rc;
        if ((rc = scratch(h, SCR_Y, (size_t)n * MLP_OUT, &ys))) return rc;
        CK(cudaMemcpyAsync(xs, X, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, h->st));
        src = xs;
        dst = ys;
    }
    MlpArgs A{};
    {
        Scope s(h->prof, "mlp_infer");
        CK(launch_mlp_infer(A, h->mlp_pk, src, dst, n, 0, h->st));
    }
    if (!on_device)
        CK(cudaMemcpyAsync(Y, dst, (size_t)n * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return RHI_OK;
}

int rhi_mlp_loss_grad(rhi_handle h, const float* X, const float* Y, long long n, float* grad,
                      double* loss, int on_device) {
    if (!h) return RHI_ERR_ARG;
    if (!h->mlp_ready) return fail(h, RHI_ERR_STATE, "rhi_mlp_loss_grad: no weights set");
    if (!X || !Y || n < 1) return fail(h, RHI_ERR_ARG, "rhi_mlp_loss_grad: bad arguments");
    const float *xs = X, *ys = Y;
    int rc;
    if (!on_device) {
        float *xd, *yd;
        if ((rc = scratch(h, SCR_X, (size_t)n * MLP_IN, &xd))) return rc;
        if ((rc = scratch(h, SCR_Y, (size_t)n * MLP_OUT, &yd))) return rc;
        CK(cudaMemcpyAsync(xd, X, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, h->st));
        CK(cudaMemcpyAsync(yd, Y, (size_t)n * MLP_OUT * sizeof(float), cudaMemcpyHostToDevice, h->st));
        xs = xd;
        ys = yd;
    }
    const long long nb = (n + mlp_train_block() - 1) / mlp_train_block();
    double* part;
    if ((rc = scratch(h, SCR_PART, (size_t)nb, &part))) return rc;
    CK(cudaMemsetAsync(h->mlp_g, 0, RHI_MLP_NWEIGHTS * sizeof(float), h->st));
    if ((rc = mlp_grad(h, xs, ys, n, part))) return rc;
    LinLaunch L(h->st, &h->prof);
    CK(L.reduce(part, (int)nb, h->scal, RED_SUM, S_TMP));
    double se = 0.0;
    if ((rc = read_scalar(h, S_TMP, &se))) return rc;
    if (loss) *loss = se / ((double)n * MLP_OUT);
    if (grad)
        CK(cudaMemcpyAsync(grad, h->mlp_g, RHI_MLP_NWEIGHTS * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    h->prof.resolve();
    return RHI_OK;
}

int rhi_mlp_train(rhi_handle h, const float* X, const float* Y, long long n, int epochs,
                  int batch, double lr, double* loss) {
    if (!h) return RHI_ERR_ARG;
    if (!h->mlp_ready) return fail(h, RHI_ERR_STATE, "rhi_mlp_train: no weights set");
    if (!X || !Y || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0))
        return fail(h, RHI_ERR_ARG, "rhi_mlp_train: bad arguments");
    const long long tb = mlp_train_block();
    const long long nbatch = (n + batch - 1) / batch;
    // block partials of one epoch, one slice per minibatch
    const long long nparts = nbatch * (((long long)batch + tb - 1) / tb);
    if (nparts > (1LL << 30)) return fail(h, RHI_ERR_ARG, "rhi_mlp_train: too many samples");
    double* part;
    int rc;
    if ((rc = scratch(h, SCR_PART, (size_t)nparts, &part))) return rc;
    CK(cudaMemsetAsync(part, 0, (size_t)nparts * sizeof(double), h->st));
    const int nupd = RHI_MLP_NWEIGHTS - 2 * RHI_MLP_IN;        // normalisation stays fixed
    for (int ep = 0; ep < epochs; ++ep) {
        long long po = 0;
        for (long long b = 0; b < nbatch; ++b) {
            const long long s0 = b * batch;
            const long long m = std::min<long long>(batch, n - s0);
            if ((rc = mlp_grad(h, X + s0 * MLP_IN, Y + s0 * MLP_OUT, m, part + po))) return rc;
            po += (m + tb - 1) / tb;
            h->mlp_t += 1;
            const float b1t = (float)std::pow(0.9, (double)h->mlp_t);
            const float b2t = (float)std::pow(0.999, (double)h->mlp_t);
            Scope s(h->prof, "mlp_adam");
            CK(launch_mlp_adam(h->mlp_w, h->mlp_g, h->mlp_m1, h->mlp_m2, nupd, (float)lr, b1t, b2t, h->st));
        }
        if (ep == epochs - 1 && loss) {
            LinLaunch L(h->st, &h->prof);
            CK(L.reduce(part, (int)po, h->scal, RED_SUM, S_TMP));
            double se = 0.0;
            if ((rc = read_scalar(h, S_TMP, &se))) return rc;
            *loss = se / ((double)n * MLP_OUT);
        }
    }
    if ((rc = mlp_repack(h))) return rc;
    h->prof.resolve();
    return RHI_OK;
}

}  // extern "C"
