// sdc_api.cu -- C ABI of libsdc (declared in include/sdc.h): context set-up,
// the SDC step driver of Eq. sdc:general (paper section 2) captured as a CUDA
// graph, and the small elementwise kernels of the path.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sdc.h"
#include "sdc_adjoint_launch.h"
#include "sdc_fourth_launch.h"
#include "sdc_launch.h"

using namespace sdcd;

namespace {

constexpr int EW_BLOCK = 256;

__global__ void set_scalar_kernel(double* p, double v) { *p = v; }

// rhs of Eq. sdc:general from elementwise arrays:
//   rhs = U^m + dtm (A^{m,(k+1)} - A^{m,(k)}) - dtm R^{m+1,(k)} + sum_l (q_l dt) (A_l + R_l)^{(k)}
// Anew_m = NULL drops the A difference (node 0, whose A never changes within a
// step, or a step with A off); the second-order path fuses the other nodes'
// rhs into the stencil kernel instead.
__global__ void rhs_kernel(int nvar, int dim, long long N, const double* __restrict__ Um,
                           const double* __restrict__ Anew_m, RhsArgs ra) {
    // one thread per zone, every field: the step's scalars once per zone
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double dt = *ra.dt;
    const double dtm = dt * ra.dtm_frac;
    double qdt[MAXM];
    for (int l = 0; l < MAXM; l++) qdt[l] = ra.qw[l] * dt;
    for (int f = 0; f < nvar; f++) {
        const long long i = (long long)f * N + z;
        const bool reactive = f >= 1 + dim;
        const long long ir = (long long)(f - 1 - dim) * N + z;
        double v = Um[i];
        if (Anew_m) v += dtm * (Anew_m[i] - ra.Aold_m[i]);
        if (reactive) v -= dtm * ra.Rnext[ir];
        double I = 0.0;
        for (int l = 0; l < ra.M; l++) {
            double src = ra.Aold[l][i];
            if (reactive) src += ra.Rold[l][ir];
            I += qdt[l] * src;
        }
        ra.rhs[i] = v + I;
    }
}

// The Newton start of the fourth-order implicit update, formed on the zone
// averages before their centre maps: the explicit predictor
// rhs + dt_m R^{m+1,(k)} (rho and rho u of the rhs, separate roundings as in
// the oracle) where it has a positive temperature and no mass fraction below
// -0.01, the previous iterate elsewhere.  out may be guess.
__global__ void predict_kernel(NetParams P, int nvar, int dim, long long N, const double* __restrict__ rhs,
                               const double* __restrict__ Rk, const double* guess, const double* __restrict__ dt,
                               double dt_frac, double* out) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= N) return;
    const double dtm = (*dt) * dt_frac;
    const double rho = rhs[z];
    double m2 = 0.0;
    for (int d = 0; d < dim; d++) m2 += rhs[(1 + d) * N + z] * rhs[(1 + d) * N + z];
    const double ir = rcp_nr(rho);
    const double wE = __dadd_rn(rhs[(1 + dim) * N + z], __dmul_rn(dtm, Rk[z]));
    const double T = P.gm1 * (wE - 0.5 * m2 * ir) * ir;
    bool ok = T > 0.0 && T < INFINITY;
    const int ns = nvar - 2 - dim;
    for (int i = 0; i < ns; i++)
        ok = ok && !(__dadd_rn(rhs[(2 + dim + i) * N + z], __dmul_rn(dtm, Rk[(1 + i) * N + z])) < -XMARGIN * rho);
    if (ok) {
        for (int f = 0; f <= dim; f++) out[f * N + z] = rhs[f * N + z];
        for (int r = 0; r <= ns; r++)
            out[(1 + dim + r) * N + z] = __dadd_rn(rhs[(1 + dim + r) * N + z], __dmul_rn(dtm, Rk[r * N + z]));
    } else if (out != guess) {
        for (int f = 0; f < nvar; f++) out[f * N + z] = guess[f * N + z];
    }
}

// I = sum_l (q_l dt) (A_l + R_l)
__global__ void node_integral_kernel(int nvar, int dim, int M, long long N, const double* __restrict__ A,
                                     const double* __restrict__ R, double q0, double q1, double q2, double q3,
                                     double dt,
                                     double* __restrict__ I) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nvar * N) return;
    const int f = (int)(i / N);
    const long long z = i - (long long)f * N;
    const int n = nvar - 1 - dim;
    const bool reactive = f >= 1 + dim;
    const int r = f - 1 - dim;
    const double q[MAXM] = {q0, q1, q2, q3};
    double s = 0.0;
    for (int l = 0; l < M; l++) {
        double src = A[(long long)l * nvar * N + i];
        if (reactive) src += R[(long long)l * n * N + r * N + z];
        s += (q[l] * dt) * src;
    }
    I[i] = s;
}

// max over zones of sum_d (|u_d| + c) / dx_d; non-negative doubles order like
// their bit patterns, so the maximum is an unsigned integer atomicMax
__global__ void cfl_kernel(NetParams P, int dim, int nbox, long long N, const BoxDev* __restrict__ boxes,
                           const double* __restrict__ U, unsigned long long* __restrict__ out) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (z < N) {
        int lo = 0, hi = nbox - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (boxes[mid].off <= z) lo = mid; else hi = mid - 1;
        }
        const BoxDev b = boxes[lo];
        const double rho = U[z];
        const double ir = 1.0 / rho;
        double u[3], ke = 0.0;
        for (int d = 0; d < dim; d++) {
            u[d] = U[(1 + d) * N + z] * ir;
            ke += 0.5 * rho * u[d] * u[d];
        }
        const double p = P.gm1 * (U[(1 + dim) * N + z] - ke);
        const double c = sqrt(P.gamma * p * ir);
        for (int d = 0; d < dim; d++) s += (fabs(u[d]) + c) * b.idx[d];
        if (!(s >= 0.0)) s = INFINITY;  // a NaN state gives no usable step
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

__global__ void selftest_math_kernel(const double* __restrict__ x, long long n, double* __restrict__ r,
                                     double* __restrict__ q) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] = rcp_nr(x[i]);
    q[i] = sqrt_nr(x[i]);
}

__global__ void selftest_pow_kernel(const double* __restrict__ T, const double* __restrict__ nu, long long n,
                                    double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = exp2_tab(nu[i] * log2_tab(T[i]));
}

constexpr int QUEUE_SLOTS = 64;

// Event pairs bracketing each launch of an eagerly enqueued step.
enum { CLS_STENCIL = 0, CLS_NEWTON = 1, CLS_OTHER = 2 };
struct Prof {
    std::vector<cudaEvent_t> ev;
    std::vector<int> cls;
    cudaStream_t st = nullptr;
    cudaError_t mark() {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
        return cudaEventRecord(e, st);
    }
    ~Prof() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// record an event before and after a launch when profiling
#define SDC_LAUNCH(prof, klass, call)                                      \
    do {                                                                   \
        if (prof && (e = prof->mark()) != cudaSuccess) return e;           \
        if ((e = (call)) != cudaSuccess) return e;                         \
        if (prof) {                                                        \
            if ((e = prof->mark()) != cudaSuccess) return e;               \
            prof->cls.push_back(klass);                                    \
        }                                                                  \
    } while (0)

}  // namespace

struct sdc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;      // borrowed
    cudaStream_t cap_stream = nullptr;  // owned: graph capture
    int nbox = 0, dim = 0, nspec = 0, nvar = 0, nw = 0;
    long long Ntot = 0;
    NetParams P;
    NewtonCfg cfg;
    int M = 0, K = 0, limiter = 1, prec = 0;
    double tau[MAXM] = {0, 0, 0, 0};
    double q[MAXM - 1][MAXM] = {{0}};
    BoxDev* d_boxes = nullptr;
    TileDev* d_tiles = nullptr;
    int ntiles = 0;
    // the direction-split stencil (3D): tiles of each pass and the primitives buffer
    TileDev* d_tiles_split[3] = {nullptr, nullptr, nullptr};
    int ntiles_split[3] = {0, 0, 0};
    double* prim = nullptr;
    double* d_dt = nullptr;
    double* node_ws[MAXM - 1] = {nullptr};    // node 0 (copy of U^n), nodes 1..M-2
    double* A0 = nullptr;                     // A at node 0 (fixed within a step)
    double* R0 = nullptr;
    double* Ag[2][MAXM] = {{nullptr}};        // two generations of A at nodes 1..M-1
    double* Rg[2][MAXM] = {{nullptr}};
    double* rhs = nullptr;
    double* anchor = nullptr;                 // the step's rate anchors (alpha chain; NewtonCfg::anchor)
    DevStats* d_stats = nullptr;
    unsigned long long* d_smax = nullptr;
    std::vector<void*> allocs;
    // the step's graphs for the last two U pointers (a caller that alternates two
    // buffers replays both), and the slot to replace next
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    double* gU[2] = {nullptr, nullptr};
    int gnext = 0;
    cudaGraphExec_t gexec_strang = nullptr;  // the Strang-split step's graph
    double* gU_strang = nullptr;
    double* d_dt_half = nullptr;             // dt/2 of the split step (next to d_dt)
    int space_order = 2;                     // 2: PLM/HLLC stencil; 4: the fourth-order operators
    FourthWs fw;                             // their workspace (space_order 4)
    // kernel variants (chosen by sdc_autotune) and the Newton work queues
    int stencil_variant = 0, newton_variant = 0;
    int persistent_blocks = 0;
    unsigned long long* d_queue = nullptr;  // one counter per Newton launch of a step
    std::vector<sdc_box> boxes;
    int tiles_capacity = 0;
    // adjoint workspace (allocated by the first sdc_step_backward)
    struct {
        bool ready = false;
        double* work = nullptr;        // the recomputed step
        std::vector<double*> store;    // U_m^{(k+1)}, k = 0..K-1, m = 1..M-1
        double* Ubar_node[MAXM] = {nullptr};
        double* Abar[2][MAXM] = {{nullptr}};
        double* Rbar[2][MAXM] = {{nullptr}};
        double *Abar_n = nullptr, *Rbar_n = nullptr, *Ubar_n = nullptr, *rhsbar = nullptr;
        double *G = nullptr, *abar_zone = nullptr;
    } adj;
};

namespace {

sdc_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SDC_OK;
    if (e == cudaErrorMemoryAllocation) return SDC_ERR_OOM;
    return SDC_ERR_CUDA;
}

#define SDC_TRY(x)                                   \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

cudaError_t ctx_alloc(sdc_ctx* c, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) c->allocs.push_back(*p);
    return e;
}

bool is_alpha_chain(const sdc_network* net) {
    if (net->nreac != net->nspec - 1 || net->nspec < 3) return false;
    for (int j = 0; j < net->nreac; j++) {
        const int* r = net->reac + 2 * j;
        const int* c = net->cnt + 2 * j;
        if (j == 0) {
            if (!(r[0] == 0 && c[0] == 3 && r[1] < 0 && net->prod[0] == 1)) return false;
        } else {
            if (!(r[0] == j && c[0] == 1 && r[1] == 0 && c[1] == 1 && net->prod[j] == j + 1)) return false;
        }
    }
    return true;
}

// Node positions (units of the step) and node-to-node weights q[m][l] of the
// integral in Eq. sdc:general.  Gauss-Lobatto: the Lagrange interpolant through
// all nodes integrated node to node (trapezoid; Simpson in two halves).
// Radau: node 0 plus the right-endpoint Gauss-Radau points, the interpolant
// through those points only (weight 0 for node 0): the Radau IIA coefficients
// as differences a_{m+1,l} - a_{m,l} (s = 1: a = 1; s = 2: a = [[5/12, -1/12],
// [3/4, 1/4]]).
void weights(int type, int M, double tau[MAXM], double q[MAXM - 1][MAXM]) {
    for (int m = 0; m < MAXM - 1; m++)
        for (int l = 0; l < MAXM; l++) q[m][l] = 0.0;
    for (int l = 0; l < MAXM; l++) tau[l] = 1.0;
    if (type == SDC_NODES_RADAU) {
        if (M == 2) {
            tau[0] = 0.0; tau[1] = 1.0; tau[2] = 1.0;
            q[0][1] = 1.0;
        } else if (M == 4) {
            // s = 3: c = (4 -/+ sqrt 6)/10, 1 and the Radau IIA coefficients
            // a_11 = (88 - 7 r)/360, a_12 = (296 - 169 r)/1800, a_13 = (-2 + 3 r)/225,
            // a_21 = (296 + 169 r)/1800, a_22 = (88 + 7 r)/360, a_23 = (-2 - 3 r)/225,
            // a_31 = (16 - r)/36, a_32 = (16 + r)/36, a_33 = 1/9 (r = sqrt 6)
            const double r = sqrt(6.0);
            const double a[3][3] = {{(88.0 - 7.0 * r) / 360.0, (296.0 - 169.0 * r) / 1800.0, (-2.0 + 3.0 * r) / 225.0},
                                    {(296.0 + 169.0 * r) / 1800.0, (88.0 + 7.0 * r) / 360.0, (-2.0 - 3.0 * r) / 225.0},
                                    {(16.0 - r) / 36.0, (16.0 + r) / 36.0, 1.0 / 9.0}};
            tau[0] = 0.0; tau[1] = (4.0 - r) / 10.0; tau[2] = (4.0 + r) / 10.0; tau[3] = 1.0;
            for (int l = 0; l < 3; l++) {
                q[0][1 + l] = a[0][l];
                q[1][1 + l] = a[1][l] - a[0][l];
                q[2][1 + l] = a[2][l] - a[1][l];
            }
        } else {
            tau[0] = 0.0; tau[1] = 1.0 / 3.0; tau[2] = 1.0;
            q[0][1] = 5.0 / 12.0; q[0][2] = -1.0 / 12.0;
            q[1][1] = 1.0 / 3.0; q[1][2] = 1.0 / 3.0;
        }
        return;
    }
    if (M == 2) {
        tau[0] = 0.0; tau[1] = 1.0; tau[2] = 1.0;
        q[0][0] = 0.5; q[0][1] = 0.5;
    } else {
        tau[0] = 0.0; tau[1] = 0.5; tau[2] = 1.0;
        q[0][0] = 5.0 / 24.0; q[0][1] = 1.0 / 3.0; q[0][2] = -1.0 / 24.0;
        q[1][0] = -1.0 / 24.0; q[1][1] = 1.0 / 3.0; q[1][2] = 5.0 / 24.0;
    }
}

// The terms of the node integral sum_l q_{m,l} (A_l + R_l): nodes with weight
// zero are left out (Radau: node 0), and nodes whose A and R are the same
// arrays (every node in the first iteration, when all hold A and R at U^n)
// become one term with the summed weight; ra.M counts the terms.
RhsArgs rhs_args(const sdc_ctx* c, const double* const* Aold, const double* const* Rold, int m,
                 const double* dt_dev) {
    RhsArgs ra;
    int nt = 0;
    for (int l = 0; l < MAXM; l++) {
        ra.Aold[l] = nullptr;
        ra.Rold[l] = nullptr;
        ra.qw[l] = 0.0;
    }
    for (int l = 0; l < c->M; l++) {
        const double w = c->q[m][l];
        if (w == 0.0) continue;
        int t = 0;
        while (t < nt && !(ra.Aold[t] == Aold[l] && ra.Rold[t] == Rold[l])) t++;
        if (t == nt) {
            ra.Aold[nt] = Aold[l];
            ra.Rold[nt] = Rold[l];
            ra.qw[nt] = 0.0;
            nt++;
        }
        ra.qw[t] += w;
    }
    ra.Rnext = Rold[m + 1];
    ra.Aold_m = Aold[m];
    ra.rhs = c->rhs;
    ra.dt = dt_dev;
    ra.dtm_frac = c->tau[m + 1] - c->tau[m];
    ra.M = nt;
    return ra;
}

// The second-order advective term of U into A (with the rhs when mode is
// STENCIL_A_RHS) by the context's stencil variant: a tile shape of
// stencil_kernel, or the direction-split passes.
cudaError_t launch_A(const sdc_ctx* c, const double* U, double* A, int mode, const RhsArgs& ra, cudaStream_t st) {
    if (c->stencil_variant == stencil_split_variant(c->dim, c->nspec))
        return launch_stencil_split(c->P, c->limiter, c->Ntot, c->d_boxes, c->d_tiles_split, c->ntiles_split, U,
                                    c->prim, A, mode, ra, st);
    return launch_stencil(c->P, c->dim, c->limiter, c->Ntot, c->d_boxes, c->d_tiles, c->ntiles, U, A, mode, ra, st,
                          c->stencil_variant);
}

// Operators of a step: both (the coupled SDC step), or one of them alone (the
// sub-problems of the Strang-split step: A = 0, or R = 0 with the implicit
// update reduced to w = rhs).
enum { OP_BOTH = 0, OP_ADVECT = 1, OP_REACT = 2 };

// Enqueue one SDC step on stream st (dt already in *dt_dev, c->d_dt by
// default); U is node M-1.  With prof, every kernel launch is bracketed by
// events (eager profiling).  reset_stats = false keeps accumulating the Newton
// statistics (the sub-steps of a split step).
cudaError_t enqueue_step(sdc_ctx* c, double* U, cudaStream_t st, Prof* prof = nullptr,
                         double* const* store = nullptr, int op = OP_BOTH, const double* dt_dev = nullptr,
                         bool reset_stats = true) {
    const long long N = c->Ntot;
    const size_t ubytes = sizeof(double) * c->nvar * N;
    const bool with_A = op != OP_REACT, with_R = op != OP_ADVECT;
    if (!dt_dev) dt_dev = c->d_dt;
    cudaError_t e;
    if (reset_stats && (e = cudaMemsetAsync(c->d_stats, 0, sizeof(DevStats), st)) != cudaSuccess) return e;
    if (c->d_queue &&
        (e = cudaMemsetAsync(c->d_queue, 0, sizeof(unsigned long long) * QUEUE_SLOTS, st)) != cudaSuccess)
        return e;
    int qslot = 0;
    double* node[MAXM];
    node[0] = c->node_ws[0];
    for (int m = 1; m < c->M - 1; m++) node[m] = c->node_ws[m];
    node[c->M - 1] = U;
    if ((e = cudaMemcpyAsync(node[0], U, ubytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    RhsArgs none = rhs_args(c, (const double* const*)c->Ag[0], (const double* const*)c->Rg[0], 0, dt_dev);
    const bool fourth = c->space_order == 4;
    if (with_A) {
        if (fourth)
            SDC_LAUNCH(prof, CLS_STENCIL, launch_advective4(c->P, c->dim, c->limiter, N, c->d_boxes, c->nbox,
                                                            node[0], c->A0, c->fw, st));
        else
            SDC_LAUNCH(prof, CLS_STENCIL, launch_A(c, node[0], c->A0, STENCIL_A, none, st));
    } else if ((e = cudaMemsetAsync(c->A0, 0, ubytes, st)) != cudaSuccess) {
        return e;
    }
    if (with_R) {
        if (fourth)
            SDC_LAUNCH(prof, CLS_OTHER, launch_reaction_source4(c->P, c->dim, N, c->d_boxes, c->nbox, node[0], c->R0,
                                                                c->fw, st));
        else
            SDC_LAUNCH(prof, CLS_OTHER, launch_reaction_source(c->P, N, c->dim, node[0], c->R0, st, c->anchor));
    } else if ((e = cudaMemsetAsync(c->R0, 0, sizeof(double) * c->nw * N, st)) != cudaSuccess) {
        return e;
    }
    const double* Aold[MAXM] = {c->A0, c->A0, c->A0, c->A0};
    const double* Rold[MAXM] = {c->R0, c->R0, c->R0, c->R0};
    // the second-order step's Newton solves take the rate anchors R(U^n) just wrote
    NewtonCfg cfg_a = c->cfg;
    cfg_a.anchor = with_R ? c->anchor : nullptr;
    for (int k = 0; k < c->K; k++) {
        const int g = k & 1;
        // an operator that is off stays zero: its arrays are all the zeroed node-0 array
        double* Anew[MAXM];
        double* Rnew[MAXM];
        Anew[0] = c->A0;
        Rnew[0] = c->R0;
        for (int m = 1; m < MAXM; m++) {
            Anew[m] = (with_A && m < c->M) ? c->Ag[g][m] : c->A0;
            Rnew[m] = (with_R && m < c->M) ? c->Rg[g][m] : c->R0;
        }
        for (int m = 0; m < c->M - 1; m++) {
            RhsArgs ra = rhs_args(c, Aold, Rold, m, dt_dev);
            if (m == 0 || !with_A) {
                // no A^{m,(k+1)} - A^{m,(k)} term: node 0 is fixed, or A is off
                SDC_LAUNCH(prof, CLS_OTHER, (rhs_kernel<<<grid_for(N, EW_BLOCK), EW_BLOCK, 0,
                                                           st>>>(c->nvar, c->dim, N, node[m], nullptr, ra),
                                             cudaGetLastError()));
            } else if (fourth) {
                SDC_LAUNCH(prof, CLS_STENCIL, launch_advective4(c->P, c->dim, c->limiter, N, c->d_boxes, c->nbox,
                                                                node[m], Anew[m], c->fw, st));
                SDC_LAUNCH(prof, CLS_OTHER, (rhs_kernel<<<grid_for(N, EW_BLOCK), EW_BLOCK, 0,
                                                           st>>>(c->nvar, c->dim, N, node[m], Anew[m], ra),
                                             cudaGetLastError()));
            } else {
                SDC_LAUNCH(prof, CLS_STENCIL, launch_A(c, node[m], Anew[m], STENCIL_A_RHS, ra, st));
            }
            if (with_R) {
                // the previous iterate U^{m+1,(k)} (U^n in the first iteration) and
                // R^{m+1,(k)}: the FP64 Newton starts from the explicit predictor
                // rhs + dt_m R^{m+1,(k)} where admissible, from that iterate
                // elsewhere.  The FP32-Jacobian solve starts from the iterate: its
                // iterative refinement stops on the same absolute step test, and
                // from the predictor that test passes after one refinement step,
                // which leaves trace species at about 1e-7 of themselves
                const double* guess = (k == 0) ? node[0] : node[m + 1];
                const double* Rpred = c->prec != SDC_PREC_FP32_JAC ? Rold[m + 1] : nullptr;
                unsigned long long* q = (c->d_queue && qslot < QUEUE_SLOTS) ? c->d_queue + qslot++ : nullptr;
                if (fourth && !Rpred) {
                    SDC_LAUNCH(prof, CLS_NEWTON, launch_newton4(c->P, c->cfg, c->prec, c->dim, N, c->d_boxes, c->nbox,
                                                                c->rhs, guess, node[m + 1], Rnew[m + 1], dt_dev,
                                                                c->tau[m + 1] - c->tau[m], 0.0, nullptr, nullptr,
                                                                c->d_stats, c->fw, st, c->newton_variant, q,
                                                                c->persistent_blocks));
                } else if (fourth) {
                    SDC_LAUNCH(prof, CLS_OTHER, (predict_kernel<<<grid_for(N, EW_BLOCK), EW_BLOCK, 0, st>>>(
                                                     c->P, c->nvar, c->dim, N, c->rhs, Rold[m + 1], guess, dt_dev,
                                                     c->tau[m + 1] - c->tau[m], node[m + 1]),
                                                 cudaGetLastError()));
                    SDC_LAUNCH(prof, CLS_NEWTON, launch_newton4(c->P, c->cfg, c->prec, c->dim, N, c->d_boxes, c->nbox,
                                                                c->rhs, node[m + 1], node[m + 1], Rnew[m + 1], dt_dev,
                                                                c->tau[m + 1] - c->tau[m], 0.0, nullptr, nullptr,
                                                                c->d_stats, c->fw, st, c->newton_variant, q,
                                                                c->persistent_blocks));
                } else
                    SDC_LAUNCH(prof, CLS_NEWTON, launch_newton(c->P, cfg_a, c->prec, N, c->dim, c->rhs, guess,
                                                               Rpred, node[m + 1], Rnew[m + 1], dt_dev,
                                                               c->tau[m + 1] - c->tau[m], 0.0, nullptr, nullptr,
                                                               c->d_stats, st, c->newton_variant, q,
                                                               c->persistent_blocks));
            } else if ((e = cudaMemcpyAsync(node[m + 1], c->rhs, ubytes, cudaMemcpyDeviceToDevice, st)) !=
                       cudaSuccess) {
                return e;  // R = 0: the implicit update is w = rhs
            }
            if (store &&
                (e = cudaMemcpyAsync(store[k * (c->M - 1) + m], node[m + 1], ubytes, cudaMemcpyDeviceToDevice, st)) !=
                    cudaSuccess)
                return e;
        }
        if (k < c->K - 1 && with_A) {
            if (fourth)
                SDC_LAUNCH(prof, CLS_STENCIL, launch_advective4(c->P, c->dim, c->limiter, N, c->d_boxes, c->nbox,
                                                                node[c->M - 1], Anew[c->M - 1], c->fw, st));
            else
                SDC_LAUNCH(prof, CLS_STENCIL, launch_A(c, node[c->M - 1], Anew[c->M - 1], STENCIL_A, none, st));
        }
        for (int l = 1; l < c->M; l++) {
            Aold[l] = Anew[l];
            Rold[l] = Rnew[l];
        }
    }
    return cudaSuccess;
}

// the captured graphs hold constants and variants: drop them after a change
void drop_graphs(sdc_ctx* c) {
    for (int i = 0; i < 2; i++) {
        if (c->gexec[i]) cudaGraphExecDestroy(c->gexec[i]);
        c->gexec[i] = nullptr;
        c->gU[i] = nullptr;
    }
    c->gnext = 0;
    if (c->gexec_strang) cudaGraphExecDestroy(c->gexec_strang);
    c->gexec_strang = nullptr;
    c->gU_strang = nullptr;
}

// stencil tiles of every box for tile shape `variant`
std::vector<TileDev> tile_list(const sdc_ctx* c, int variant) {
    std::vector<TileDev> ht;
    int tl[3];
    stencil_tile(c->dim, c->nspec, variant, tl);
    for (int b = 0; b < (int)c->boxes.size(); b++)
        for (int z = 0; z < c->boxes[b].n[2]; z += tl[2])
            for (int y = 0; y < c->boxes[b].n[1]; y += tl[1])
                for (int x = 0; x < c->boxes[b].n[0]; x += tl[0]) ht.push_back(TileDev{b, {x, y, z}});
    return ht;
}

// tiles of direction-split pass D of every box
std::vector<TileDev> split_tile_list(const sdc_ctx* c, int D) {
    std::vector<TileDev> ht;
    int tl[3];
    split_tile_shape(D, tl);
    for (int b = 0; b < (int)c->boxes.size(); b++)
        for (int z = 0; z < c->boxes[b].n[2]; z += tl[2])
            for (int y = 0; y < c->boxes[b].n[1]; y += tl[1])
                for (int x = 0; x < c->boxes[b].n[0]; x += tl[0]) ht.push_back(TileDev{b, {x, y, z}});
    return ht;
}

cudaError_t set_stencil_variant(sdc_ctx* c, int variant) {
    if (variant == stencil_split_variant(c->dim, c->nspec)) {
        if (!c->prim) return cudaErrorInvalidValue;  // a context without the split workspace
        c->stencil_variant = variant;
        return cudaSuccess;
    }
    std::vector<TileDev> ht = tile_list(c, variant);
    if ((int)ht.size() > c->tiles_capacity) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpy(c->d_tiles, ht.data(), sizeof(TileDev) * ht.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    c->ntiles = (int)ht.size();
    c->stencil_variant = variant;
    return cudaSuccess;
}

void stats_to_host(const DevStats& d, sdc_stats* s) {
    s->newton_iters_total = (long long)d.iters_total;
    s->newton_solves = (long long)d.solves;
    s->n_fail = (long long)d.fails;
    for (int i = 0; i < 64; i++) s->hist[i] = (long long)d.hist[i];
}

sdc_status read_stats(sdc_ctx* c, sdc_stats* stats) {
    DevStats h;
    SDC_TRY(cudaMemcpyAsync(&h, c->d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
    SDC_TRY(cudaStreamSynchronize(c->stream));
    stats_to_host(h, stats);
    return stats->n_fail ? SDC_ERR_NEWTON_NOCONV : SDC_OK;
}

// the adjoint workspace of the context, allocated on first use
cudaError_t adjoint_workspace(sdc_ctx* c) {
    auto& A = c->adj;
    if (A.ready) return cudaSuccess;
    const long long N = c->Ntot;
    const int M = c->M, K = c->K, nw = c->nw, nr = c->P.nreac;
    const size_t ub = sizeof(double) * c->nvar * N, rb = sizeof(double) * nw * N;
    cudaError_t e;
#define ADJ_ALLOC(ptr, bytes) \
    if ((e = ctx_alloc(c, (void**)&(ptr), (bytes))) != cudaSuccess) return e;
    ADJ_ALLOC(A.work, ub);
    A.store.assign(K * (M - 1), nullptr);
    for (auto& p : A.store) ADJ_ALLOC(p, ub);
    for (int m = 0; m < M; m++) ADJ_ALLOC(A.Ubar_node[m], ub);
    for (int g = 0; g < 2; g++)
        for (int m = 0; m < M; m++) {
            ADJ_ALLOC(A.Abar[g][m], ub);
            ADJ_ALLOC(A.Rbar[g][m], rb);
        }
    ADJ_ALLOC(A.Abar_n, ub);
    ADJ_ALLOC(A.Rbar_n, rb);
    ADJ_ALLOC(A.Ubar_n, ub);
    ADJ_ALLOC(A.rhsbar, ub);
    ADJ_ALLOC(A.G, sizeof(double) * (size_t)c->dim * N * 4 * c->nvar);
    ADJ_ALLOC(A.abar_zone, sizeof(double) * (size_t)(nr > 0 ? nr : 1) * N);
#undef ADJ_ALLOC
    A.ready = true;
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char* sdc_status_string(sdc_status s) {
    switch (s) {
        case SDC_OK: return "ok";
        case SDC_ERR_INVALID_ARG: return "invalid argument";
        case SDC_ERR_CUDA: return "CUDA error";
        case SDC_ERR_OOM: return "out of device memory";
        case SDC_ERR_NEWTON_NOCONV: return "Newton iteration did not converge in some zones";
        case SDC_ERR_NONPHYSICAL: return "no admissible Newton step in some zones";
        case SDC_ERR_TIMEOUT: return "bounded device wait expired";
        case SDC_ERR_TOO_LARGE: return "problem exceeds the static scratch of sdc_step_static (48 MiB)";
    }
    return "unknown status";
}

void sdc_destroy(sdc_ctx* ctx) {
    if (!ctx) return;
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (void* p : ctx->allocs) cudaFree(p);
    delete ctx;
}

sdc_status sdc_init_box(const sdc_box* boxes, int nbox, const sdc_network* net, const sdc_params* prm,
                        void* cuda_stream, sdc_ctx** out) {
    if (!out) return SDC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!boxes || nbox < 1 || !net || !prm) return SDC_ERR_INVALID_ARG;
    const int dim = boxes[0].dim;
    if (dim != 1 && dim != 3) return SDC_ERR_INVALID_ARG;
    long long Ntot = 0;
    for (int b = 0; b < nbox; b++) {
        if (boxes[b].dim != dim) return SDC_ERR_INVALID_ARG;
        for (int d = 0; d < 3; d++) {
            if (boxes[b].n[d] < 1) return SDC_ERR_INVALID_ARG;
            if (d >= dim && boxes[b].n[d] != 1) return SDC_ERR_INVALID_ARG;
            if (d < dim && !(boxes[b].dx[d] > 0.0)) return SDC_ERR_INVALID_ARG;
        }
        const long long nb = (long long)boxes[b].n[0] * boxes[b].n[1] * boxes[b].n[2];
        if (nb >= (1ll << 31)) return SDC_ERR_INVALID_ARG;  // zone indices inside a box are 32-bit
        Ntot += nb;
    }
    if (net->nspec < 1 || net->nspec > SDC_MAX_SPEC || net->nreac < 1 || net->nreac > SDC_MAX_REAC)
        return SDC_ERR_INVALID_ARG;
    if (!net->mass || !net->a || !net->nu || !net->Q || !net->reac || !net->cnt || !net->prod)
        return SDC_ERR_INVALID_ARG;
    if (net->rate_law != SDC_RATE_POWER && net->rate_law != SDC_RATE_ARRHENIUS) return SDC_ERR_INVALID_ARG;
    for (int j = 0; j < net->nreac; j++) {
        for (int s = 0; s < 2; s++) {
            const int sp = net->reac[2 * j + s];
            if (sp >= net->nspec || sp < -1) return SDC_ERR_INVALID_ARG;
            if (sp >= 0 && (net->cnt[2 * j + s] < 1 || net->cnt[2 * j + s] > 3)) return SDC_ERR_INVALID_ARG;
        }
        if (net->reac[2 * j] < 0) return SDC_ERR_INVALID_ARG;
        if (net->reac[2 * j] == net->reac[2 * j + 1]) return SDC_ERR_INVALID_ARG;
        if (net->prod[j] < 0 || net->prod[j] >= net->nspec) return SDC_ERR_INVALID_ARG;
    }
    if (!(prm->gamma > 1.0) || prm->n_nodes < 2 || prm->n_nodes > 3 + (prm->node_type == SDC_NODES_RADAU) ||
        prm->n_iters < 1 ||
        prm->newton_maxit < 1 || !(prm->newton_rtol > 0.0) ||
        (prm->prec != SDC_PREC_FP64 && prm->prec != SDC_PREC_FP32_JAC && prm->prec != SDC_PREC_FP32X2_JAC) ||
        (prm->node_type != SDC_NODES_LOBATTO && prm->node_type != SDC_NODES_RADAU) ||
        (prm->space_order != 2 && prm->space_order != 4))
        return SDC_ERR_INVALID_ARG;
    const int topo = is_alpha_chain(net) ? TOPO_CHAIN : TOPO_GENERIC;
    int topo_used = topo;
    if (!newton_supported(net->nspec, topo_used)) {
        topo_used = TOPO_GENERIC;
        if (!newton_supported(net->nspec, topo_used)) return SDC_ERR_INVALID_ARG;
    }
    // the float-pair matrix: the alpha chain's bordered form only
    if (prm->prec == SDC_PREC_FP32X2_JAC && topo_used != TOPO_CHAIN) return SDC_ERR_INVALID_ARG;
    // the per-thread rate arrays hold nspec - 1 reactions
    if (net->nreac > net->nspec - 1) return SDC_ERR_INVALID_ARG;
    if (!stencil_supported(dim, net->nspec)) return SDC_ERR_INVALID_ARG;

    sdc_ctx* c = new (std::nothrow) sdc_ctx();
    if (!c) return SDC_ERR_OOM;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->nbox = nbox;
    c->dim = dim;
    c->nspec = net->nspec;
    c->nvar = 2 + dim + net->nspec;
    c->nw = net->nspec + 1;
    c->Ntot = Ntot;
    c->M = prm->n_nodes;
    c->K = prm->n_iters;
    c->limiter = prm->limiter ? 1 : 0;
    c->prec = prm->prec;
    c->newton_variant = newton_default_variant(net->nspec, topo_used, prm->prec);
    c->cfg.rtol = prm->newton_rtol;
    c->cfg.maxit = prm->newton_maxit;
    c->space_order = prm->space_order;
    weights(prm->node_type, c->M, c->tau, c->q);
    NetParams& P = c->P;
    memset(&P, 0, sizeof(P));
    P.nspec = net->nspec;
    P.nreac = net->nreac;
    P.law = net->rate_law;
    P.topo = topo_used;
    P.gamma = prm->gamma;
    P.gm1 = prm->gamma - 1.0;
    P.gm1_inv = 1.0 / P.gm1;
    for (int i = 0; i < net->nspec; i++) {
        P.mass[i] = net->mass[i];
        P.inv_mass[i] = 1.0 / net->mass[i];
    }
    for (int j = 0; j < net->nreac; j++) {
        P.a[j] = net->a[j];
        P.nu[j] = net->nu[j];
        P.Q[j] = net->Q[j];
        P.r0[j] = net->reac[2 * j];
        P.c0[j] = net->cnt[2 * j];
        P.r1[j] = net->reac[2 * j + 1];
        P.c1[j] = net->reac[2 * j + 1] >= 0 ? net->cnt[2 * j + 1] : 0;
        P.prod[j] = net->prod[j];
        P.order[j] = P.c0[j] + P.c1[j];
    }
    set_chain_coefs(P);

    // boxes and stencil tiles (the tile table is sized for the smallest tile shape)
    std::vector<BoxDev> hb(nbox);
    long long off = 0;
    for (int b = 0; b < nbox; b++) {
        hb[b].off = off;
        for (int d = 0; d < 3; d++) {
            hb[b].n[d] = boxes[b].n[d];
            hb[b].idx[d] = d < dim ? 1.0 / boxes[b].dx[d] : 0.0;
        }
        off += (long long)boxes[b].n[0] * boxes[b].n[1] * boxes[b].n[2];
    }
    c->boxes.assign(boxes, boxes + nbox);
    int max_tiles = 0;
    for (int v = 0; v < stencil_variants(dim, net->nspec); v++) {
        if (v == stencil_split_variant(dim, net->nspec)) continue;
        const int nt = (int)tile_list(c, v).size();
        if (nt > max_tiles) max_tiles = nt;
    }
    c->tiles_capacity = max_tiles;
    std::vector<TileDev> ht = tile_list(c, 0);
    c->ntiles = (int)ht.size();

    sdc_status st = SDC_OK;
    auto fail = [&](cudaError_t e) {
        sdc_destroy(c);
        return cuda_status(e);
    };
    cudaError_t e;
    if ((e = stencil_prepare(dim, net->nspec)) != cudaSuccess) return fail(e);
    if ((e = newton_prepare(net->nspec, topo_used)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->d_boxes, sizeof(BoxDev) * nbox)) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->d_tiles, sizeof(TileDev) * c->tiles_capacity)) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->d_queue, sizeof(unsigned long long) * QUEUE_SLOTS)) != cudaSuccess) return fail(e);
    c->persistent_blocks = newton_persistent_blocks(P, c->prec);
    if ((e = ctx_alloc(c, (void**)&c->d_dt, 2 * sizeof(double))) != cudaSuccess) return fail(e);
    c->d_dt_half = c->d_dt + 1;
    if ((e = ctx_alloc(c, (void**)&c->d_stats, sizeof(DevStats))) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->d_smax, sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    const size_t ub = sizeof(double) * c->nvar * Ntot, rb = sizeof(double) * c->nw * Ntot;
    if ((e = ctx_alloc(c, (void**)&c->node_ws[0], ub)) != cudaSuccess) return fail(e);
    for (int m = 1; m < c->M - 1; m++)
        if ((e = ctx_alloc(c, (void**)&c->node_ws[m], ub)) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->A0, ub)) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->R0, rb)) != cudaSuccess) return fail(e);
    if ((e = ctx_alloc(c, (void**)&c->rhs, ub)) != cudaSuccess) return fail(e);
    if (c->P.topo == TOPO_CHAIN && c->space_order == 2 &&
        (e = ctx_alloc(c, (void**)&c->anchor, sizeof(double) * (size_t)(c->P.nreac + 2) * Ntot)) != cudaSuccess)
        return fail(e);
    if (dim == 3 && c->space_order == 2) {
        // the direction-split stencil: the primitives buffer and the tiles of its passes
        if ((e = ctx_alloc(c, (void**)&c->prim, ub)) != cudaSuccess) return fail(e);
        for (int D = 0; D < 3; D++) {
            std::vector<TileDev> st3 = split_tile_list(c, D);
            c->ntiles_split[D] = (int)st3.size();
            if ((e = ctx_alloc(c, (void**)&c->d_tiles_split[D], sizeof(TileDev) * st3.size())) != cudaSuccess)
                return fail(e);
            if ((e = cudaMemcpy(c->d_tiles_split[D], st3.data(), sizeof(TileDev) * st3.size(),
                                cudaMemcpyHostToDevice)) != cudaSuccess)
                return fail(e);
        }
    }
    for (int g = 0; g < 2; g++)
        for (int m = 1; m < c->M; m++) {
            if ((e = ctx_alloc(c, (void**)&c->Ag[g][m], ub)) != cudaSuccess) return fail(e);
            if ((e = ctx_alloc(c, (void**)&c->Rg[g][m], rb)) != cudaSuccess) return fail(e);
        }
    if (c->space_order == 4) {
        FourthWs& w = c->fw;
        double** arrays[] = {&w.Uc, &w.W2, &w.Wc, &w.Wa, &w.Fc, &w.F2, &w.Fa, &w.rc, &w.gc};
        for (double** a : arrays)
            if ((e = ctx_alloc(c, (void**)a, ub)) != cudaSuccess) return fail(e);
        // the face states: one face average and its centre map (smooth form) or
        // the two limited sides (limited form)
        double** faces[] = {c->limiter ? &w.WL : &w.Wf, c->limiter ? &w.WR : &w.Wfc};
        for (double** a : faces)
            if ((e = ctx_alloc(c, (void**)a, ub)) != cudaSuccess) return fail(e);
        if ((e = ctx_alloc(c, (void**)&w.Rc, rb)) != cudaSuccess) return fail(e);
    }
    if ((e = cudaMemcpy(c->d_boxes, hb.data(), sizeof(BoxDev) * nbox, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemcpy(c->d_tiles, ht.data(), sizeof(TileDev) * ht.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemset(c->d_stats, 0, sizeof(DevStats))) != cudaSuccess) return fail(e);
    (void)st;
    *out = c;
    return SDC_OK;
}

sdc_status sdc_sizes(const sdc_ctx* ctx, long long* ntot, int* nvar, int* nreactive) {
    if (!ctx) return SDC_ERR_INVALID_ARG;
    if (ntot) *ntot = ctx->Ntot;
    if (nvar) *nvar = ctx->nvar;
    if (nreactive) *nreactive = ctx->nw;
    return SDC_OK;
}

sdc_status sdc_advective_term(sdc_ctx* ctx, const double* U, double* A) {
    if (!ctx || !U || !A || U == A) return SDC_ERR_INVALID_ARG;
    if (ctx->space_order == 4) {
        SDC_TRY(launch_advective4(ctx->P, ctx->dim, ctx->limiter, ctx->Ntot, ctx->d_boxes, ctx->nbox, U, A, ctx->fw,
                                  ctx->stream));
        return SDC_OK;
    }
    RhsArgs none;
    memset(&none, 0, sizeof(none));
    SDC_TRY(launch_A(ctx, U, A, STENCIL_A, none, ctx->stream));
    return SDC_OK;
}

sdc_status sdc_node_integral(sdc_ctx* ctx, const double* A_nodes, const double* R_nodes, double dt, int m,
                             double* I) {
    if (!ctx || !A_nodes || !R_nodes || !I || m < 0 || m >= ctx->M - 1) return SDC_ERR_INVALID_ARG;
    const long long n = (long long)ctx->nvar * ctx->Ntot;
    node_integral_kernel<<<grid_for(n, EW_BLOCK), EW_BLOCK, 0, ctx->stream>>>(
        ctx->nvar, ctx->dim, ctx->M, ctx->Ntot, A_nodes, R_nodes, ctx->q[m][0], ctx->q[m][1], ctx->q[m][2], ctx->q[m][3], dt, I);
    SDC_TRY(cudaGetLastError());
    return SDC_OK;
}

sdc_status sdc_react_newton(sdc_ctx* ctx, const double* rhs, double dt_m, double* U_inout, double* R_out,
                            int* zone_status, int* zone_iters, sdc_stats* stats) {
    if (!ctx || !rhs || !U_inout || !R_out || rhs == U_inout) return SDC_ERR_INVALID_ARG;
    if (stats) SDC_TRY(cudaMemsetAsync(ctx->d_stats, 0, sizeof(DevStats), ctx->stream));
    SDC_TRY(cudaMemsetAsync(ctx->d_queue, 0, sizeof(unsigned long long), ctx->stream));
    if (ctx->space_order == 4)
        SDC_TRY(launch_newton4(ctx->P, ctx->cfg, ctx->prec, ctx->dim, ctx->Ntot, ctx->d_boxes, ctx->nbox, rhs, U_inout,
                               U_inout, R_out, nullptr, 1.0, dt_m, zone_status, zone_iters, ctx->d_stats, ctx->fw,
                               ctx->stream, ctx->newton_variant, ctx->d_queue, ctx->persistent_blocks));
    else
        SDC_TRY(launch_newton(ctx->P, ctx->cfg, ctx->prec, ctx->Ntot, ctx->dim, rhs, U_inout, nullptr, U_inout, R_out,
                              nullptr, 1.0, dt_m, zone_status, zone_iters, ctx->d_stats, ctx->stream,
                              ctx->newton_variant, ctx->d_queue, ctx->persistent_blocks));
    if (stats) return read_stats(ctx, stats);
    return SDC_OK;
}

sdc_status sdc_step(sdc_ctx* ctx, double* U, double dt, sdc_stats* stats) {
    if (!ctx || !U || !(dt > 0.0)) return SDC_ERR_INVALID_ARG;
    int slot = -1;
    for (int i = 0; i < 2; i++)
        if (ctx->gexec[i] && ctx->gU[i] == U) slot = i;
    if (slot < 0) {
        slot = ctx->gnext;
        if (ctx->gexec[slot]) {
            cudaGraphExecDestroy(ctx->gexec[slot]);
            ctx->gexec[slot] = nullptr;
            ctx->gU[slot] = nullptr;
        }
        cudaGraph_t graph = nullptr;
        SDC_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_step(ctx, U, ctx->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_status(e != cudaSuccess ? e : e2);
        }
        e = cudaGraphInstantiate(&ctx->gexec[slot], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->gexec[slot] = nullptr;
            return cuda_status(e);
        }
        ctx->gU[slot] = U;
    }
    ctx->gnext = 1 - slot;  // the other graph is the one replaced next
    set_scalar_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_dt, dt);
    SDC_TRY(cudaGetLastError());
    SDC_TRY(cudaGraphLaunch(ctx->gexec[slot], ctx->stream));
    if (stats) return read_stats(ctx, stats);
    return SDC_OK;
}

sdc_status sdc_step_strang(sdc_ctx* ctx, double* U, double dt, sdc_stats* stats) {
    if (!ctx || !U || !(dt > 0.0)) return SDC_ERR_INVALID_ARG;
    if (!ctx->gexec_strang || ctx->gU_strang != U) {
        if (ctx->gexec_strang) {
            cudaGraphExecDestroy(ctx->gexec_strang);
            ctx->gexec_strang = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaStream_t cs = ctx->cap_stream;
        SDC_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(ctx->d_stats, 0, sizeof(DevStats), cs);
        if (e == cudaSuccess) e = enqueue_step(ctx, U, cs, nullptr, nullptr, OP_REACT, ctx->d_dt_half, false);
        if (e == cudaSuccess) e = enqueue_step(ctx, U, cs, nullptr, nullptr, OP_ADVECT, ctx->d_dt, false);
        if (e == cudaSuccess) e = enqueue_step(ctx, U, cs, nullptr, nullptr, OP_REACT, ctx->d_dt_half, false);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_status(e != cudaSuccess ? e : e2);
        }
        e = cudaGraphInstantiate(&ctx->gexec_strang, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->gexec_strang = nullptr;
            return cuda_status(e);
        }
        ctx->gU_strang = U;
    }
    set_scalar_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_dt, dt);
    SDC_TRY(cudaGetLastError());
    set_scalar_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_dt_half, 0.5 * dt);
    SDC_TRY(cudaGetLastError());
    SDC_TRY(cudaGraphLaunch(ctx->gexec_strang, ctx->stream));
    if (stats) return read_stats(ctx, stats);
    return SDC_OK;
}

sdc_status sdc_step_profile(sdc_ctx* ctx, double* U, double dt, sdc_stats* stats, sdc_profile* prof) {
    if (!ctx || !U || !(dt > 0.0) || !prof) return SDC_ERR_INVALID_ARG;
    memset(prof, 0, sizeof(*prof));
    Prof P;
    P.st = ctx->stream;
    set_scalar_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_dt, dt);
    SDC_TRY(cudaGetLastError());
    SDC_TRY(enqueue_step(ctx, U, ctx->stream, &P));
    SDC_TRY(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < P.cls.size(); i++) {
        float ms = 0.0f;
        SDC_TRY(cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]));
        if (P.cls[i] == CLS_STENCIL) { prof->launches_stencil++; prof->ms_stencil += ms; }
        else if (P.cls[i] == CLS_NEWTON) { prof->launches_newton++; prof->ms_newton += ms; }
        else { prof->launches_other++; prof->ms_other += ms; }
    }
    prof->launches_other++;  // the kernel that stores dt
    if (stats) return read_stats(ctx, stats);
    return SDC_OK;
}

sdc_status sdc_selftest_math(const double* x, long long n, double* rcp_out, double* sqrt_out, void* cuda_stream) {
    if (!x || !rcp_out || !sqrt_out || n < 0) return SDC_ERR_INVALID_ARG;
    if (n == 0) return SDC_OK;
    selftest_math_kernel<<<grid_for(n, EW_BLOCK), EW_BLOCK, 0, (cudaStream_t)cuda_stream>>>(x, n, rcp_out, sqrt_out);
    SDC_TRY(cudaGetLastError());
    return SDC_OK;
}

sdc_status sdc_selftest_pow(const double* T, const double* nu, long long n, double* out, void* cuda_stream) {
    if (!T || !nu || !out || n < 0) return SDC_ERR_INVALID_ARG;
    if (n == 0) return SDC_OK;
    selftest_pow_kernel<<<grid_for(n, EW_BLOCK), EW_BLOCK, 0, (cudaStream_t)cuda_stream>>>(T, nu, n, out);
    SDC_TRY(cudaGetLastError());
    return SDC_OK;
}

sdc_status sdc_autotune(sdc_ctx* ctx, const double* U, double dt, sdc_tuning* out) {
    if (!ctx || !U || !(dt > 0.0)) return SDC_ERR_INVALID_ARG;
    const size_t ub = sizeof(double) * ctx->nvar * ctx->Ntot;
    double* scratch = nullptr;
    SDC_TRY(cudaMalloc((void**)&scratch, ub));
    sdc_tuning t;
    memset(&t, 0, sizeof(t));
    t.stencil_variants = stencil_variants(ctx->dim, ctx->nspec);
    t.newton_variants = newton_variants(ctx->nspec, ctx->P.topo);
    if (t.stencil_variants > SDC_MAX_VARIANTS || t.newton_variants > SDC_MAX_VARIANTS) {
        cudaFree(scratch);
        return SDC_ERR_INVALID_ARG;
    }
    sdc_status st = SDC_OK;
    // one eager step per candidate (after one warm-up step); the step's stencil
    // time depends only on the tile shape and its Newton time only on the
    // Newton variant, so each is chosen on its own
    auto trial = [&](float* ms_st, float* ms_nw) -> sdc_status {
        sdc_profile pr;
        for (int rep = 0; rep < 2; rep++) {
            if (cudaMemcpyAsync(scratch, U, ub, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
                return SDC_ERR_CUDA;
            sdc_status s2 = sdc_step_profile(ctx, scratch, dt, nullptr, &pr);
            if (s2 != SDC_OK && s2 != SDC_ERR_NEWTON_NOCONV) return s2;
        }
        *ms_st = pr.ms_stencil;
        *ms_nw = pr.ms_newton;
        return SDC_OK;
    };
    const int nv0 = ctx->newton_variant;
    float best_st = 0.0f, best_nw = 0.0f;
    int vs = 0, vn = 0;
    for (int v = 0; v < t.stencil_variants && st == SDC_OK; v++) {
        // the fourth-order operators use no tile shape, and their contexts hold
        // no workspace for the direction-split passes
        if (v == stencil_split_variant(ctx->dim, ctx->nspec) && !ctx->prim) continue;
        if (set_stencil_variant(ctx, v) != cudaSuccess) { st = SDC_ERR_CUDA; break; }
        float a, b;
        st = trial(&a, &b);
        t.ms_stencil[v] = a;
        if (st == SDC_OK && (v == 0 || a < best_st)) { best_st = a; vs = v; }
    }
    bool first_nw = true;
    for (int v = 0; v < t.newton_variants && st == SDC_OK; v++) {
        if (!newton_variant_ok(ctx->nspec, ctx->P.topo, ctx->prec, v)) continue;  // not built for this precision
        ctx->newton_variant = v;
        float a, b;
        st = trial(&a, &b);
        t.ms_newton[v] = b;
        if (st == SDC_OK && (first_nw || b < best_nw)) { best_nw = b; vn = v; first_nw = false; }
    }
    cudaFree(scratch);
    if (st != SDC_OK) {
        ctx->newton_variant = nv0;
        set_stencil_variant(ctx, 0);
        return st;
    }
    SDC_TRY(set_stencil_variant(ctx, vs));
    ctx->newton_variant = vn;
    t.stencil_choice = vs;
    t.newton_choice = vn;
    // the captured graph used the previous variants
    drop_graphs(ctx);
    if (out) *out = t;
    return SDC_OK;
}

sdc_status sdc_set_variants(sdc_ctx* ctx, int stencil_variant, int newton_variant) {
    if (!ctx || stencil_variant < 0 || stencil_variant >= stencil_variants(ctx->dim, ctx->nspec) ||
        !newton_variant_ok(ctx->nspec, ctx->P.topo, ctx->prec, newton_variant))
        return SDC_ERR_INVALID_ARG;
    if (stencil_variant == stencil_split_variant(ctx->dim, ctx->nspec) && !ctx->prim) return SDC_ERR_INVALID_ARG;
    SDC_TRY(set_stencil_variant(ctx, stencil_variant));
    ctx->newton_variant = newton_variant;
    drop_graphs(ctx);
    return SDC_OK;
}

sdc_status sdc_launches_per_step(const sdc_ctx* ctx, int* launches) {
    if (!ctx || !launches) return SDC_ERR_INVALID_ARG;
    // dt store, A(U^n), R(U^n), per iteration and node a rhs kernel and a Newton
    // kernel, and A at the last node for every iteration but the last
    if (ctx->space_order == 4) {
        // fourth order: A is a sequence of kernels and is evaluated apart from
        // the rhs at nodes m >= 1; the source and the implicit update add maps
        const int LA = fourth_advective_launches(ctx->dim, ctx->limiter), K = ctx->K, M = ctx->M;
        const int predict = ctx->prec != SDC_PREC_FP32_JAC ? 1 : 0;  // the predictor start's kernel
        *launches = 1 + LA + FOURTH_SOURCE_LAUNCHES + K * (M - 1) * (1 + predict + FOURTH_NEWTON_LAUNCHES) +
                    K * (M - 2) * LA + (K - 1) * LA;
        return SDC_OK;
    }
    *launches = 3 + ctx->K * 2 * (ctx->M - 1) + (ctx->K - 1);
    if (ctx->stencil_variant == stencil_split_variant(ctx->dim, ctx->nspec)) {
        // three passes per advective term: A(U^n), the fused rhs at nodes 1..M-2,
        // and A at the last node for every iteration but the last
        const int evals = 1 + ctx->K * (ctx->M - 2) + (ctx->K - 1);
        *launches += 2 * evals;
    }
    return SDC_OK;
}

sdc_status sdc_set_rates(sdc_ctx* ctx, const double* a) {
    if (!ctx || !a) return SDC_ERR_INVALID_ARG;
    for (int j = 0; j < ctx->P.nreac; j++) ctx->P.a[j] = a[j];
    set_chain_coefs(ctx->P);  // the chain's prefactors a_j / prod mass
    drop_graphs(ctx);  // the captured graphs hold the old constants
    return SDC_OK;
}

sdc_status sdc_advective_term_vjp(sdc_ctx* ctx, const double* U, const double* Abar, double* Ubar, int mode) {
    if (!ctx || !U || !Abar || !Ubar || (mode != 0 && mode != 1)) return SDC_ERR_INVALID_ARG;
    if (!adjoint_supported(ctx->dim, ctx->nspec, ctx->P.topo) || ctx->space_order != 2) return SDC_ERR_INVALID_ARG;
    SDC_TRY(adjoint_workspace(ctx));
    SDC_TRY(launch_stencil_vjp(ctx->P, ctx->dim, ctx->limiter, ctx->Ntot, ctx->d_boxes, ctx->nbox, U, Abar,
                               ctx->adj.G, Ubar, ctx->stream, mode));
    return SDC_OK;
}

sdc_status sdc_step_backward(sdc_ctx* ctx, const double* U_n, double dt, const double* gU_np1, double* gU_n,
                             double* g_a) {
    if (!ctx || !U_n || !gU_np1 || !gU_n || !(dt > 0.0)) return SDC_ERR_INVALID_ARG;
    if (!adjoint_supported(ctx->dim, ctx->nspec, ctx->P.topo) || ctx->space_order != 2) return SDC_ERR_INVALID_ARG;
    sdc_ctx* c = ctx;
    const long long N = c->Ntot;
    const int M = c->M, K = c->K, nw = c->nw, nr = c->P.nreac;
    const size_t ub = sizeof(double) * c->nvar * N, rb = sizeof(double) * nw * N;
    cudaStream_t st = c->stream;
    auto& A = c->adj;
    SDC_TRY(adjoint_workspace(c));
    // 1. recompute the step from the checkpoint, keeping every node state
    SDC_TRY(cudaMemcpyAsync(A.work, U_n, ub, cudaMemcpyDeviceToDevice, st));
    set_scalar_kernel<<<1, 1, 0, st>>>(c->d_dt, dt);
    SDC_TRY(cudaGetLastError());
    SDC_TRY(enqueue_step(c, A.work, st, nullptr, A.store.data()));
    // 2. reverse sweep
    for (int m = 0; m < M; m++) SDC_TRY(cudaMemsetAsync(A.Ubar_node[m], 0, ub, st));
    for (int g = 0; g < 2; g++)
        for (int m = 0; m < M; m++) {
            SDC_TRY(cudaMemsetAsync(A.Abar[g][m], 0, ub, st));
            SDC_TRY(cudaMemsetAsync(A.Rbar[g][m], 0, rb, st));
        }
    SDC_TRY(cudaMemsetAsync(A.Abar_n, 0, ub, st));
    SDC_TRY(cudaMemsetAsync(A.Rbar_n, 0, rb, st));
    SDC_TRY(cudaMemsetAsync(A.Ubar_n, 0, ub, st));
    SDC_TRY(cudaMemsetAsync(A.abar_zone, 0, sizeof(double) * (size_t)(nr > 0 ? nr : 1) * N, st));
    SDC_TRY(cudaMemcpyAsync(A.Ubar_node[M - 1], gU_np1, ub, cudaMemcpyDeviceToDevice, st));
    int gnew = 0, gold = 1;
    for (int k = K - 1; k >= 0; k--) {
        double *Aold[MAXM], *Rold[MAXM];
        for (int l = 0; l < MAXM; l++) {
            const bool un = (l == 0 || k == 0);  // values at U^n
            Aold[l] = un ? A.Abar_n : A.Abar[gold][l];
            Rold[l] = un ? A.Rbar_n : A.Rbar[gold][l];
        }
        auto Ust = [&](int m) { return A.store[k * (M - 1) + (m - 1)]; };  // U_m^{(k+1)}, m >= 1
        if (k < K - 1)
            SDC_TRY(launch_stencil_vjp(c->P, c->dim, c->limiter, N, c->d_boxes, c->nbox, Ust(M - 1),
                                       A.Abar[gnew][M - 1], A.G, A.Ubar_node[M - 1], st));
        for (int m = M - 2; m >= 0; m--) {
            const double dtm = dt * (c->tau[m + 1] - c->tau[m]);
            SDC_TRY(launch_reaction_vjp(c->P, c->dim, N, Ust(m + 1), A.Rbar[gnew][m + 1], A.Ubar_node[m + 1], dtm,
                                        A.rhsbar, A.abar_zone, st));
            RhsAdjArgs ra;
            memset(&ra, 0, sizeof(ra));
            ra.nvar = c->nvar;
            ra.dim = c->dim;
            ra.M = M;
            ra.m = m;
            ra.N = N;
            ra.rhsbar = A.rhsbar;
            ra.Ubar_m = m >= 1 ? A.Ubar_node[m] : A.Ubar_n;
            ra.Abar_new_m = m >= 1 ? A.Abar[gnew][m] : nullptr;
            for (int l = 0; l < MAXM; l++) {
                ra.Abar_old[l] = Aold[l];
                ra.Rbar_old[l] = Rold[l];
                ra.qdt[l] = c->q[m][l] * dt;
            }
            ra.dtm = dtm;
            SDC_TRY(launch_rhs_adjoint(ra, st));
            if (m >= 1)
                SDC_TRY(launch_stencil_vjp(c->P, c->dim, c->limiter, N, c->d_boxes, c->nbox, Ust(m), A.Abar[gnew][m],
                                           A.G, A.Ubar_node[m], st));
        }
        // the adjoints of this iteration's inputs are the next ones' outputs
        const int t = gnew;
        gnew = gold;
        gold = t;
        for (int m = 0; m < M; m++) {
            SDC_TRY(cudaMemsetAsync(A.Abar[gold][m], 0, ub, st));
            SDC_TRY(cudaMemsetAsync(A.Rbar[gold][m], 0, rb, st));
        }
        for (int m = 1; m < M; m++) SDC_TRY(cudaMemsetAsync(A.Ubar_node[m], 0, ub, st));
    }
    // A(U^n) and R(U^n)
    SDC_TRY(launch_stencil_vjp(c->P, c->dim, c->limiter, N, c->d_boxes, c->nbox, U_n, A.Abar_n, A.G, A.Ubar_n, st));
    SDC_TRY(launch_reaction_vjp(c->P, c->dim, N, U_n, A.Rbar_n, A.Ubar_n, 0.0, nullptr, A.abar_zone, st));
    SDC_TRY(cudaMemcpyAsync(gU_n, A.Ubar_n, ub, cudaMemcpyDeviceToDevice, st));
    if (g_a) SDC_TRY(launch_reduce_rows(N, nr, A.abar_zone, g_a, st));
    return SDC_OK;
}

sdc_status sdc_cfl_dt(sdc_ctx* ctx, const double* U, double cfl, double* dt_out) {
    if (!ctx || !U || !dt_out || !(cfl > 0.0)) return SDC_ERR_INVALID_ARG;
    SDC_TRY(cudaMemsetAsync(ctx->d_smax, 0, sizeof(unsigned long long), ctx->stream));
    cfl_kernel<<<grid_for(ctx->Ntot, EW_BLOCK), EW_BLOCK, 0, ctx->stream>>>(ctx->P, ctx->dim, ctx->nbox, ctx->Ntot,
                                                                           ctx->d_boxes, U, ctx->d_smax);
    SDC_TRY(cudaGetLastError());
    unsigned long long bits = 0;
    SDC_TRY(cudaMemcpyAsync(&bits, ctx->d_smax, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
    SDC_TRY(cudaStreamSynchronize(ctx->stream));
    double smax;
    memcpy(&smax, &bits, sizeof(smax));
    if (!(smax > 0.0) || !(smax < INFINITY)) return SDC_ERR_NONPHYSICAL;
    *dt_out = cfl / smax;
    return SDC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sdc_step_static: one SDC step whose workspace lives in a fixed device array,
// for callers that cannot allocate device memory.  In host code the array's
// name is only a host-side stand-in: its device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) unsigned char g_static_scratch[SDC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int STATIC_MAX_DEVICES = 64;
std::mutex g_static_mutex;
void* g_static_ptr[STATIC_MAX_DEVICES] = {nullptr};

// device address of the scratch array on the current device
cudaError_t static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

struct StaticTables {
    int nbox;
    int t[3];                                   // stencil tile
    long long off[SDC_STATIC_MAX_BOXES];
    int n[SDC_STATIC_MAX_BOXES][3];
    double idx[SDC_STATIC_MAX_BOXES][3];
    int tile_first[SDC_STATIC_MAX_BOXES + 1];   // prefix sum of tiles per box
};

// box table and tile list written into the scratch array
__global__ void static_tables_kernel(StaticTables T, BoxDev* boxes, TileDev* tiles) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T.nbox) {
        boxes[i].off = T.off[i];
        for (int d = 0; d < 3; d++) {
            boxes[i].n[d] = T.n[i][d];
            boxes[i].idx[d] = T.idx[i][d];
        }
    }
    if (i >= T.tile_first[T.nbox]) return;
    int b = 0;
    while (b + 1 < T.nbox && T.tile_first[b + 1] <= i) b++;
    const int local = i - T.tile_first[b];
    const int nx = (T.n[b][0] + T.t[0] - 1) / T.t[0], ny = (T.n[b][1] + T.t[1] - 1) / T.t[1];
    TileDev td;
    td.box = b;
    td.o[0] = (local % nx) * T.t[0];
    td.o[1] = ((local / nx) % ny) * T.t[1];
    td.o[2] = (local / (nx * ny)) * T.t[2];
    tiles[i] = td;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" sdc_status sdc_step_static(const sdc_box* boxes, int nbox, const sdc_network* net, const sdc_params* prm,
                                      void* cuda_stream, double* U, double dt, sdc_stats* stats) {
    if (!boxes || nbox < 1 || nbox > SDC_STATIC_MAX_BOXES || !net || !prm || !U || !(dt > 0.0))
        return SDC_ERR_INVALID_ARG;
    const int dim = boxes[0].dim;
    if (dim != 1 && dim != 3) return SDC_ERR_INVALID_ARG;
    if (net->nspec < 1 || net->nspec > SDC_MAX_SPEC || net->nreac < 1 || net->nreac > net->nspec - 1)
        return SDC_ERR_INVALID_ARG;
    if (!net->mass || !net->a || !net->nu || !net->Q || !net->reac || !net->cnt || !net->prod)
        return SDC_ERR_INVALID_ARG;
    if (net->rate_law != SDC_RATE_POWER && net->rate_law != SDC_RATE_ARRHENIUS) return SDC_ERR_INVALID_ARG;
    for (int j = 0; j < net->nreac; j++) {
        for (int s = 0; s < 2; s++) {
            const int sp = net->reac[2 * j + s];
            if (sp >= net->nspec || sp < -1) return SDC_ERR_INVALID_ARG;
            if (sp >= 0 && (net->cnt[2 * j + s] < 1 || net->cnt[2 * j + s] > 3)) return SDC_ERR_INVALID_ARG;
        }
        if (net->reac[2 * j] < 0 || net->reac[2 * j] == net->reac[2 * j + 1]) return SDC_ERR_INVALID_ARG;
        if (net->prod[j] < 0 || net->prod[j] >= net->nspec) return SDC_ERR_INVALID_ARG;
    }
    if (!(prm->gamma > 1.0) || (prm->n_nodes != 2 && prm->n_nodes != 3) || prm->n_iters < 1 ||
        prm->newton_maxit < 1 || !(prm->newton_rtol > 0.0) ||
        (prm->prec != SDC_PREC_FP64 && prm->prec != SDC_PREC_FP32_JAC && prm->prec != SDC_PREC_FP32X2_JAC) ||
        (prm->node_type != SDC_NODES_LOBATTO && prm->node_type != SDC_NODES_RADAU) ||
        (prm->space_order != 2 && prm->space_order != 4))
        return SDC_ERR_INVALID_ARG;
    if (prm->space_order != 2) return SDC_ERR_INVALID_ARG;  // the fixed scratch holds the second-order step
    int topo = is_alpha_chain(net) ? TOPO_CHAIN : TOPO_GENERIC;
    if (!newton_supported(net->nspec, topo)) {
        topo = TOPO_GENERIC;
        if (!newton_supported(net->nspec, topo)) return SDC_ERR_INVALID_ARG;
    }
    if (prm->prec == SDC_PREC_FP32X2_JAC && topo != TOPO_CHAIN) return SDC_ERR_INVALID_ARG;
    if (!stencil_supported(dim, net->nspec)) return SDC_ERR_INVALID_ARG;

    // tables and sizes (stack only)
    StaticTables T;
    memset(&T, 0, sizeof(T));
    T.nbox = nbox;
    stencil_tile(dim, net->nspec, 0, T.t);
    long long Ntot = 0;
    for (int b = 0; b < nbox; b++) {
        if (boxes[b].dim != dim) return SDC_ERR_INVALID_ARG;
        for (int d = 0; d < 3; d++) {
            if (boxes[b].n[d] < 1 || (d >= dim && boxes[b].n[d] != 1)) return SDC_ERR_INVALID_ARG;
            if (d < dim && !(boxes[b].dx[d] > 0.0)) return SDC_ERR_INVALID_ARG;
            T.n[b][d] = boxes[b].n[d];
            T.idx[b][d] = d < dim ? 1.0 / boxes[b].dx[d] : 0.0;
        }
        // zone indices inside a box are 32-bit: refuse 2^31 zones or more before
        // any product can overflow (each factor is below 2^31)
        const long long n01 = (long long)boxes[b].n[0] * boxes[b].n[1];
        if (n01 >= (1ll << 31)) return SDC_ERR_TOO_LARGE;
        const long long nb = n01 * boxes[b].n[2];
        if (nb >= (1ll << 31)) return SDC_ERR_TOO_LARGE;
        T.off[b] = Ntot;
        Ntot += nb;
        // one double per zone must fit before the workspace offsets are formed
        if (Ntot > (long long)(SDC_STATIC_SCRATCH_BYTES / sizeof(double))) return SDC_ERR_TOO_LARGE;
        const long long nt = (long long)((boxes[b].n[0] + T.t[0] - 1) / T.t[0]) *
                             ((boxes[b].n[1] + T.t[1] - 1) / T.t[1]) * ((boxes[b].n[2] + T.t[2] - 1) / T.t[2]);
        if ((long long)T.tile_first[b] + nt > (1ll << 30)) return SDC_ERR_TOO_LARGE;
        T.tile_first[b + 1] = T.tile_first[b] + (int)nt;
    }
    const int nvar = 2 + dim + net->nspec, nw = net->nspec + 1, M = prm->n_nodes;
    const size_t ub = sizeof(double) * (size_t)nvar * Ntot, rb = sizeof(double) * (size_t)nw * Ntot;
    size_t off = 0;
    const size_t o_dt = off; off = align256(off + sizeof(double));
    const size_t o_stats = off; off = align256(off + sizeof(DevStats));
    const size_t o_boxes = off; off = align256(off + sizeof(BoxDev) * nbox);
    const size_t o_tiles = off; off = align256(off + sizeof(TileDev) * (size_t)T.tile_first[nbox]);
    size_t o_node[2], o_A0, o_R0, o_rhs, o_Ag[2][3] = {{0}}, o_Rg[2][3] = {{0}};
    o_node[0] = off; off = align256(off + ub);
    o_node[1] = off; if (M == 3) off = align256(off + ub);
    o_A0 = off; off = align256(off + ub);
    o_R0 = off; off = align256(off + rb);
    o_rhs = off; off = align256(off + ub);
    for (int g = 0; g < 2; g++)
        for (int m = 1; m < M; m++) {
            o_Ag[g][m] = off; off = align256(off + ub);
            o_Rg[g][m] = off; off = align256(off + rb);
        }
    if (off > SDC_STATIC_SCRATCH_BYTES) return SDC_ERR_TOO_LARGE;

    unsigned char* base = nullptr;
    SDC_TRY(static_scratch((void**)&base));
    SDC_TRY(stencil_prepare(dim, net->nspec));
    SDC_TRY(newton_prepare(net->nspec, topo));

    // a context on the stack whose pointers all lie inside the scratch array
    sdc_ctx c;
    c.stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c.device);
    c.nbox = nbox;
    c.dim = dim;
    c.nspec = net->nspec;
    c.nvar = nvar;
    c.nw = nw;
    c.Ntot = Ntot;
    c.M = M;
    c.K = prm->n_iters;
    c.limiter = prm->limiter ? 1 : 0;
    c.prec = prm->prec;
    c.newton_variant = newton_default_variant(net->nspec, topo, prm->prec);
    c.cfg.rtol = prm->newton_rtol;
    c.cfg.maxit = prm->newton_maxit;
    weights(prm->node_type, M, c.tau, c.q);
    NetParams& P = c.P;
    memset(&P, 0, sizeof(P));
    P.nspec = net->nspec;
    P.nreac = net->nreac;
    P.law = net->rate_law;
    P.topo = topo;
    P.gamma = prm->gamma;
    P.gm1 = prm->gamma - 1.0;
    P.gm1_inv = 1.0 / P.gm1;
    for (int i = 0; i < net->nspec; i++) {
        P.mass[i] = net->mass[i];
        P.inv_mass[i] = 1.0 / net->mass[i];
    }
    for (int j = 0; j < net->nreac; j++) {
        P.a[j] = net->a[j];
        P.nu[j] = net->nu[j];
        P.Q[j] = net->Q[j];
        P.r0[j] = net->reac[2 * j];
        P.c0[j] = net->cnt[2 * j];
        P.r1[j] = net->reac[2 * j + 1];
        P.c1[j] = net->reac[2 * j + 1] >= 0 ? net->cnt[2 * j + 1] : 0;
        P.prod[j] = net->prod[j];
        P.order[j] = P.c0[j] + P.c1[j];
    }
    set_chain_coefs(P);
    c.d_dt = (double*)(base + o_dt);
    c.d_stats = (DevStats*)(base + o_stats);
    c.d_boxes = (BoxDev*)(base + o_boxes);
    c.d_tiles = (TileDev*)(base + o_tiles);
    c.ntiles = T.tile_first[nbox];
    c.node_ws[0] = (double*)(base + o_node[0]);
    c.node_ws[1] = M == 3 ? (double*)(base + o_node[1]) : nullptr;
    c.A0 = (double*)(base + o_A0);
    c.R0 = (double*)(base + o_R0);
    c.rhs = (double*)(base + o_rhs);
    for (int g = 0; g < 2; g++)
        for (int m = 1; m < M; m++) {
            c.Ag[g][m] = (double*)(base + o_Ag[g][m]);
            c.Rg[g][m] = (double*)(base + o_Rg[g][m]);
        }
    const int nt = c.ntiles > nbox ? c.ntiles : nbox;
    static_tables_kernel<<<grid_for(nt, EW_BLOCK), EW_BLOCK, 0, c.stream>>>(T, c.d_boxes, c.d_tiles);
    SDC_TRY(cudaGetLastError());
    set_scalar_kernel<<<1, 1, 0, c.stream>>>(c.d_dt, dt);
    SDC_TRY(cudaGetLastError());
    SDC_TRY(enqueue_step(&c, U, c.stream));
    if (stats) return read_stats(&c, stats);
    return SDC_OK;
}
