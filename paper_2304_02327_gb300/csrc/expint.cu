// Orchestration: the PHISPLIT Tucker chain (Section 3, P_l^(2)) and the time
// steppers of Section 3.2 (eq. (17)-(20)), as stream-ordered launches of the
// contraction kernels (FP64: dgemm.cu, TF32x3: tf32.cu) and the prepass.
//
// Per step the big tensor makes d passes per Tucker.  Intermediates ping-pong
// between two N-double buffers; the last mode's epilogue performs the
// integrator's update in FP64 (U+ = U + tau*Y, the ETD2RK stage values and
// g(U2) - g(U)), so no separate elementwise pass touches HBM.
//
// expint_step captures its nsteps steps once per argument set into a CUDA graph
// (on a stream of the plan) and replays it, so a call costs one graph launch of
// host time whatever the number of kernels.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "plan.cuh"
#include "stencil.cuh"
#include "tf32.cuh"
#include "trace.cuh"

namespace mm {

PointwiseG pointwise_of(const mm_nonlin* g) {
    PointwiseG pg{};
    pg.kind = MM_G_NONE;
    if (!g) return pg;
    if (g->kind == MM_G_CUBIC || g->kind == MM_G_ADR_MANUFACTURED) {
        pg.kind = g->kind;
        pg.c0 = g->c[0]; pg.c1 = g->c[1]; pg.c2 = g->c[2]; pg.c3 = g->c[3];
        pg.f0 = (float)g->c[0]; pg.f1 = (float)g->c[1]; pg.f2 = (float)g->c[2]; pg.f3 = (float)g->c[3];
        pg.psi_a = g->psi_a; pg.psi_b = g->psi_b;
    }
    return pg;
}

namespace {

double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

// FP64 Tucker chain with the matrices M[0..d-1]: modes 1..d-1 store into
// outs[0..d-2]; mode d applies `last`.
int fp64_chain_m(mm_plan_s* p, const double* const* M, const double* in, double* const* outs, const Epi& last,
                 cudaStream_t s) {
    const double* cur = in;
    for (int mu = 1; mu <= p->d; ++mu) {
        Epi e{};
        if (mu < p->d) {
            e.kind = EPI_STORE;
            e.alpha = 1.0;
            e.C = outs[mu - 1];
        } else {
            e = last;
        }
        int rc = launch_dgemm(mode_gemm(p->d, p->n, mu, M[mu - 1], cur), e, s);
        if (rc) return rc;
        cur = mu < p->d ? outs[mu - 1] : nullptr;
    }
    return MM_OK;
}

// The same with the plan's phi_ell(tau A_mu).
int fp64_chain(mm_plan_s* p, int ell, const double* in, double* const* outs, const Epi& last,
               cudaStream_t s) {
    const double* M[MM_MAX_D];
    for (int mu = 0; mu < p->d; ++mu) M[mu] = p->phi[mu][ell];
    return fp64_chain_m(p, M, in, outs, last, s);
}

// J = A + X (n*n elements) and J = A + T^T (n x n): the Riccati Jacobian's directions.
__global__ void add_kernel(const double* __restrict__ A, const double* __restrict__ X, double* J, int64_t nn) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
        J[i] = A[i] + X[i];
}
__global__ void add_transpose_kernel(const double* __restrict__ A, const double* __restrict__ T, double* J, int n) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % n, c = i / n;
        J[i] = A[i] + T[c + (int64_t)n * r];
    }
}

// Tucker of `in` (consumable, N doubles) with scratch (N doubles) and the final
// epilogue `last`.  The FP64 chain ping-pongs between in and scratch.
int run_tucker(mm_plan_s* p, int ell, double* in, double* scratch, const Epi& last, cudaStream_t s) {
    double* outs[MM_MAX_D];
    for (int k = 0; k < p->d - 1; ++k) outs[k] = (k % 2 == 0) ? scratch : in;
    return fp64_chain(p, ell, in, outs, last, s);
}

// The FP64 buffer (in or scratch) that run_tucker leaves untouched while its last
// mode runs, so the last epilogue may write into it.
double* free_during_last(const mm_plan_s* p, double* in, double* scratch) {
    if (p->d == 1) return scratch;
    // FP64: the last mode reads outs[d-2] = (d-2 even ? scratch : in)
    return (p->d % 2 == 0) ? in : scratch;
}

StencilArgs stencil_base(const mm_plan_s* p, const double* U, double* W, int mode, double t,
                         const PointwiseG& pg) {
    StencilArgs a{};
    a.mode = mode; a.d = p->d; a.N = p->N;
    int64_t st = 1;
    for (int mu = 0; mu < p->d; ++mu) {
        a.n[mu] = p->n[mu];
        a.stride[mu] = st;
        st *= p->n[mu];
        a.diag3[mu] = p->diag3[mu];
    }
    a.U = U; a.W = W; a.t = t; a.g = pg;
    return a;
}

// Plain n x n-type GEMM C = A*B (+ D1*beta + D2*gamma), column-major.
int plain_gemm(int M, int N, int K, const double* A, int64_t lda, const double* B, int64_t ldb,
               double* C, int64_t ldc, const double* D1, double beta, const double* D2, double gamma,
               cudaStream_t s) {
    Gemm g{};
    g.M = M; g.N = N; g.K = K; g.batch = 1;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.b_kcontig = 1; g.ldc = ldc;
    Epi e{};
    e.kind = EPI_STORE; e.alpha = 1.0; e.C = C;
    e.D1 = D1; e.beta = beta; e.D2 = D2; e.gamma = gamma;
    return launch_dgemm(g, e, s);
}

// Riccati G(U) = C + (U B) U (eq. (2)) with U the n1 x n2 matrix view (column-major,
// n1 = riccati_rows): XB = U B, G = XB U + C + gamma*D2.
int riccati_g(const mm_plan_s* p, const mm_nonlin* g, const double* U, double* XB, double* G,
              const double* D2, double gamma, cudaStream_t s) {
    const int n1 = (int)riccati_rows(p), n2 = (int)(p->N / n1);
    int rc = plain_gemm(n1, n1, n2, U, n1, g->B, n2, XB, n1, nullptr, 0, nullptr, 0, s);
    if (rc) return rc;
    return plain_gemm(n1, n2, n1, XB, n1, U, n1, G, n1, g->C, 1.0, D2, gamma, s);
}

// W = K U + G(t, U).  For Riccati, G is also left in Gn.
int ku_plus_g(mm_plan_s* p, const mm_nonlin* g, const double* U, double t, double* W, double* Gn,
              double* XB, cudaStream_t s) {
    const PointwiseG pg = pointwise_of(g);
    const bool riccati = g && g->kind == MM_G_RICCATI;
    int rc;
    if (riccati) {
        rc = riccati_g(p, g, U, XB, Gn, nullptr, 0.0, s);
        if (rc) return rc;
    } else if (p->tridiag) {
        return launch_prepass(stencil_base(p, U, W, PRE_KU_G, t, pg), s);
    } else {
        rc = launch_prepass(stencil_base(p, U, W, PRE_G, t, pg), s);
        if (rc) return rc;
    }
    // dense K u accumulated into W: W = U x_1 A_1 + (Gn or W), then W += U x_mu A_mu
    for (int mu = 1; mu <= p->d; ++mu) {
        Gemm gm = mode_gemm(p->d, p->n, mu, p->A[mu - 1], U);
        Epi e{};
        e.kind = EPI_STORE; e.alpha = 1.0; e.C = W;
        e.D1 = (mu == 1 && riccati) ? Gn : W;
        e.beta = 1.0;
        rc = launch_dgemm(gm, e, s);
        if (rc) return rc;
    }
    return MM_OK;
}

// Rosenbrock-Euler (d = 2) workspace beyond the Riccati pieces, in doubles:
// J1 (n1^2), J2 and B U (n2^2 each), phi_0 and phi_1 of both directions, the
// phi formation's scratch (4 nmax^2), its column sums (nmax) and band word.
size_t rosenbrock_extra(const mm_plan_s* p) {
    const size_t n1 = (size_t)p->n[0], n2 = (size_t)p->n[1], nm = n1 > n2 ? n1 : n2;
    return 3 * n1 * n1 + 4 * n2 * n2 + 4 * nm * nm + nm + 2;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return a && b && x < y + nb && y < x + na;
}

int scheme_ell(int scheme) {
    switch (scheme) {
    case MM_EXPEULER: return 1;
    case MM_ETD2RK: return 2;
    case MM_LAWSON_EULER: return 0;
    case MM_LAWSON2B: return 0;
    case MM_EXPROSEULER: return 1;
    case MM_EXPEULER_ALT: return 1;
    default: return -1;
    }
}

}  // namespace

}  // namespace mm

using namespace mm;

namespace {

int run_steps(mm_plan p, int scheme, const mm_nonlin* g, double* U, double t0, int nsteps, void* ws,
              cudaStream_t s);

constexpr int kGraphSteps = 32;     // most steps one captured graph holds

bool same_nonlin(const mm_nonlin* a, int has_a, const mm_nonlin& b, int has_b) {
    if (has_a != has_b) return false;
    if (!has_a) return true;
    if (a->kind != b.kind || a->B != b.B || a->C != b.C || a->psi_a != b.psi_a || a->psi_b != b.psi_b)
        return false;
    for (int i = 0; i < 4; ++i)
        if (a->c[i] != b.c[i]) return false;
    return true;
}

// The cached graph for these arguments, if any.
const mm_graph_cache* find_graph(mm_plan p, int scheme, const mm_nonlin* g, double* U, double t0, int nsteps,
                                 void* ws) {
    const bool tdep = g && g->kind == MM_G_ADR_MANUFACTURED;
    for (const auto& e : p->graphs)
        if (e.scheme == scheme && e.nsteps == nsteps && e.U == U && e.ws == ws && same_nonlin(g, g != nullptr, e.g, e.has_g) &&
            (!tdep || e.t0 == t0))
            return &e;
    return nullptr;
}

// Capture the nsteps steps on the plan's own stream into a new cache entry (the
// oldest of more than eight is dropped).
int capture_steps(mm_plan p, int scheme, const mm_nonlin* g, double* U, double t0, int nsteps, void* ws) {
    if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
        p->cap = nullptr;
        return MM_ERR_CUDA;
    }
    mm_graph_cache e;
    e.scheme = scheme; e.nsteps = nsteps; e.U = U; e.ws = ws; e.t0 = t0;
    e.has_g = g != nullptr;
    if (g) e.g = *g;
    trace_capture_begin();
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        trace_capture_end(e.launches);
        return MM_ERR_CUDA;
    }
    const int rc = run_steps(p, scheme, g, U, t0, nsteps, ws, p->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->cap, &graph);
    trace_capture_end(e.launches);
    if (rc || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc ? rc : MM_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return MM_ERR_CUDA;
    if (p->graphs.size() >= 8) {
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back(e);
    return MM_OK;
}

}  // namespace

extern "C" int phi_plan_set_graphs(mm_plan p, int on) {
    if (!p) return MM_ERR_ARG;
    p->use_graphs = on != 0;
    return MM_OK;
}

extern "C" size_t mumode_workspace_bytes(mm_plan p) {
    if (!p) return 0;
    if (p->prec != MM_FP64) return mixed_mumode_workspace_bytes(p);
    return p->d >= 2 ? (size_t)p->N * sizeof(double) : 0;
}

extern "C" int mumode_phi_apply(mm_plan p, int ell, const double* V, double* P, double alpha,
                                void* ws, size_t ws_bytes, void* stream) {
    NvtxScope nv("mumode_phi_apply");
    if (!p || !V || !P || ell < 0 || ell > p->ell_max || !isfinite(alpha)) return MM_ERR_ARG;
    const size_t bytes = (size_t)p->N * sizeof(double);
    if (overlaps(V, bytes, P, bytes)) return MM_ERR_ARG;
    const size_t need = mumode_workspace_bytes(p);
    // the mixed forms address their operand buffers with TMA: 16-byte alignment
    const uintptr_t amask = p->prec == MM_FP64 ? 7 : 15;
    if (need && (!ws || ws_bytes < need || ((uintptr_t)ws & amask))) return MM_ERR_WORKSPACE;
    if (need && (overlaps(ws, need, V, bytes) || overlaps(ws, need, P, bytes))) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double* T = (double*)ws;
    Epi last{};
    last.kind = EPI_STORE;
    last.alpha = alpha * pow(factorial(ell), p->d - 1);
    last.C = P;
    if (p->prec != MM_FP64) {
        // split V into the mode-1 operand parts, then the tensor-core chain
        const size_t S = part_set_bytes(p);
        uint8_t* w = (uint8_t*)ws;
        int rc = mixed_split_input(p, V, w, s);
        if (rc) return rc;
        return mixed_tucker(p, ell, w, w + S, w + 2 * S, (float*)(w + 3 * S), last, s);
    }
    double* outs[MM_MAX_D];
    // mode d writes P; mode d-1 writes T; earlier modes alternate backwards
    for (int k = 0; k < p->d - 1; ++k) outs[k] = ((p->d - 2 - k) % 2 == 0) ? T : P;
    return fp64_chain(p, ell, V, outs, last, s);
}

extern "C" size_t expint_workspace_bytes(mm_plan p, int scheme, const mm_nonlin* g) {
    if (!p) return 0;
    if (p->prec != MM_FP64) return mixed_workspace_bytes(p, scheme, g ? g->kind : MM_G_NONE);
    const size_t N = (size_t)p->N;
    size_t buffers = 2;                          // Tucker ping-pong X, Y
    if (scheme == MM_ETD2RK) buffers = 3;        // + U2
    if (scheme == MM_EXPEULER_ALT) buffers = 3;  // + the first Tucker's result
    if (scheme == MM_LAWSON2B) buffers = 4;      // + Z, U2
    size_t elems = buffers * N;
    if (g && g->kind == MM_G_RICCATI && p->d % 2 == 0) {
        const size_t n1 = (size_t)riccati_rows(p);
        elems += N + (n1 * n1 > N ? n1 * n1 : N);  // Gn, XB
    }
    if (scheme == MM_EXPROSEULER && p->d == 2) elems += rosenbrock_extra(p);
    return elems * sizeof(double);
}

extern "C" int expint_step(mm_plan p, int scheme, const mm_nonlin* g, double* U, double t0,
                           int nsteps, void* ws, size_t ws_bytes, void* stream) {
    NvtxScope nv("expint_step");
    if (!p || !U || nsteps < 0 || !isfinite(t0)) return MM_ERR_ARG;
    const int ell = scheme_ell(scheme);
    if (ell < 0) return MM_ERR_ARG;
    if (ell > p->ell_max) return MM_ERR_ARG;
    const int gk = g ? g->kind : MM_G_NONE;
    if (gk < MM_G_NONE || gk > MM_G_ADR_MANUFACTURED) return MM_ERR_ARG;
    if (gk == MM_G_RICCATI) {
        // the state must have a matrix view: an even number of directions
        if (p->d % 2 != 0 || !g->B || !g->C) return MM_ERR_ARG;
        if (riccati_rows(p) > 0x7fffffffLL || p->N / riccati_rows(p) > 0x7fffffffLL) return MM_ERR_SHAPE;
        if (scheme != MM_EXPEULER && scheme != MM_ETD2RK && scheme != MM_EXPROSEULER) return MM_ERR_UNSUPPORTED;
    }
    // the Jacobian A + dG is a Kronecker sum only in the two-direction form
    if (scheme == MM_EXPROSEULER && (gk != MM_G_RICCATI || p->prec != MM_FP64 || p->d != 2))
        return MM_ERR_UNSUPPORTED;
    if (scheme == MM_EXPEULER_ALT && (gk == MM_G_RICCATI || p->prec != MM_FP64)) return MM_ERR_UNSUPPORTED;
    if (gk == MM_G_ADR_MANUFACTURED && (!g->psi_a || !g->psi_b)) return MM_ERR_ARG;
    const size_t need = expint_workspace_bytes(p, scheme, g);
    const uintptr_t amask = p->prec == MM_FP64 ? 7 : 15;
    if (!ws || ws_bytes < need || ((uintptr_t)ws & amask)) return MM_ERR_WORKSPACE;
    const size_t bytes = (size_t)p->N * sizeof(double);
    if (overlaps(ws, need, U, bytes)) return MM_ERR_ARG;
    if (nsteps == 0) return MM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // Rosenbrock-Euler forms phi of its Jacobian every step, choosing the scaling on
    // the host: it runs with direct launches only
    if (!p->use_graphs || trace_timing_on() || scheme == MM_EXPROSEULER)
        return run_steps(p, scheme, g, U, t0, nsteps, ws, s);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return run_steps(p, scheme, g, U, t0, nsteps, ws, s);      // the caller is capturing
    // Graphs hold at most kGraphSteps steps: longer calls replay that chunk (g without
    // time dependence) or launch directly (a time-dependent g bakes t into the nodes).
    const bool tdep = g && g->kind == MM_G_ADR_MANUFACTURED;
    if (nsteps > kGraphSteps && tdep) return run_steps(p, scheme, g, U, t0, nsteps, ws, s);
    for (int done = 0; done < nsteps;) {
        const int k = std::min(kGraphSteps, nsteps - done);
        const mm_graph_cache* e = find_graph(p, scheme, g, U, t0, k, ws);
        if (!e) {
            int rc = capture_steps(p, scheme, g, U, t0, k, ws);
            if (rc) return rc;
            e = &p->graphs.back();
        }
        MM_CUDA_TRY(cudaGraphLaunch(e->exec, s));
        for (int c = 0; c < MM_KC_COUNT; ++c) trace_count(c, e->launches[c]);
        done += k;
    }
    return MM_OK;
}

namespace {

// The body of expint_step after its argument checks (nsteps >= 1).
int run_steps(mm_plan p, int scheme, const mm_nonlin* g, double* U, double t0, int nsteps, void* ws,
              cudaStream_t s) {
    const int gk = g ? g->kind : MM_G_NONE;
    if (p->prec != MM_FP64) {
        return mixed_expint(p, scheme, g, U, t0, nsteps, (uint8_t*)ws, s);
    }
    const int64_t N = p->N;
    double* X = (double*)ws;
    double* Y = X + N;
    double* U2 = Y + N;                                     // ETD2RK, Lawson2b
    double* Z = (scheme == MM_LAWSON2B) ? U2 + N : nullptr; // Lawson2b second input
    double* extra = X + (scheme == MM_ETD2RK || scheme == MM_EXPEULER_ALT ? 3 : (scheme == MM_LAWSON2B ? 4 : 2)) * N;
    double* Gn = extra;                                     // Riccati
    double* XB = extra + N;
    const PointwiseG pg = pointwise_of(g);
    const double tau = p->tau;
    const int d = p->d;
    int rc = MM_OK;

    for (int k = 0; k < nsteps && rc == MM_OK; ++k) {
        const double t = t0 + k * tau;
        switch (scheme) {
        case MM_EXPEULER: {
            rc = ku_plus_g(p, g, U, t, X, Gn, XB, s);
            if (rc) break;
            Epi e{};
            e.kind = EPI_EE; e.alpha = tau; e.U = U; e.status = p->status;
            rc = run_tucker(p, 1, X, Y, e, s);
            break;
        }
        case MM_ETD2RK: {
            rc = ku_plus_g(p, g, U, t, X, Gn, XB, s);
            if (rc) break;
            double* freebuf = free_during_last(p, X, Y);
            Epi e1{};
            e1.U = U; e1.U2 = U2; e1.alpha = tau; e1.t0 = t; e1.t1 = t + tau; e1.g = pg;
            e1.status = p->status;
            double* W2 = freebuf;
            if (gk == MM_G_RICCATI) {
                e1.kind = EPI_ETD_S1_NOG;
            } else {
                e1.kind = EPI_ETD_S1;
                e1.W2 = W2;
            }
            rc = run_tucker(p, 1, X, Y, e1, s);
            if (rc) break;
            if (gk == MM_G_RICCATI) {
                // W2 = G(U2) - G(U) = (U2 B) U2 + C - Gn
                rc = riccati_g(p, g, U2, XB, W2, Gn, -1.0, s);
                if (rc) break;
            }
            double* other = (W2 == X) ? Y : X;
            Epi e2{};
            e2.kind = EPI_ETD_S2; e2.alpha = tau * pow(2.0, d - 1); e2.U = U; e2.U2 = U2;
            e2.status = p->status;
            rc = run_tucker(p, 2, W2, other, e2, s);
            break;
        }
        case MM_EXPEULER_ALT: {
            // Z = U x_mu e^{tau A_mu} (from a copy of U, which the chain consumes), then
            // U = tau G(U) x_mu phi_1(tau A_mu) + Z in the last epilogue
            double* Z = U2;
            MM_CUDA_TRY(cudaMemcpyAsync(X, U, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s));
            Epi e0{};
            e0.kind = EPI_STORE; e0.alpha = 1.0; e0.C = Z;
            rc = run_tucker(p, 0, X, Y, e0, s);
            if (rc) break;
            rc = launch_prepass(stencil_base(p, U, X, PRE_G, t, pg), s);
            if (rc) break;
            Epi e1{};
            e1.kind = EPI_STORE; e1.alpha = tau; e1.C = U; e1.D1 = Z; e1.beta = 1.0;
            rc = run_tucker(p, 1, X, Y, e1, s);
            break;
        }
        case MM_EXPROSEULER: {
            // W = K U + G(U) (and XB = U B), then J_1 = A_1 + U B, J_2 = A_2 + (B U)^T
            rc = ku_plus_g(p, g, U, t, X, Gn, XB, s);
            if (rc) break;
            const int n1 = (int)p->n[0], n2 = (int)p->n[1];
            const int64_t q1 = (int64_t)n1 * n1, q2 = (int64_t)n2 * n2;
            const int nm = n1 > n2 ? n1 : n2;
            double* J1 = XB + (q1 > N ? q1 : N);
            double* J2 = J1 + q1;
            double* BU = J2 + q2;
            double* P1[2] = {BU + q2, BU + q2 + q1};            // phi_0, phi_1 of J_1
            double* P2[2] = {P1[1] + q1, P1[1] + q1 + q2};      // of J_2
            double* scratch = P2[1] + q2;                        // 4 nm^2
            // the pieces end at scratch + 4 nm^2 + nm + 2 doubles: rosenbrock_extra()
            double* colsum = scratch + 4 * (int64_t)nm * nm;
            int* band = (int*)(colsum + nm);
            add_kernel<<<(unsigned)std::min<int64_t>((q1 + 255) / 256, 4096), 256, 0, s>>>(p->A[0], XB, J1, q1);
            rc = plain_gemm(n2, n2, n1, g->B, n2, U, n1, BU, n2, nullptr, 0, nullptr, 0, s);
            if (rc) break;
            add_transpose_kernel<<<(unsigned)std::min<int64_t>((q2 + 255) / 256, 4096), 256, 0, s>>>(p->A[1], BU,
                                                                                                   J2, n2);
            if (cudaGetLastError() != cudaSuccess) { rc = MM_ERR_CUDA; break; }
            int sq = 0, bw = 0;
            rc = form_phis(n1, J1, tau, 1, P1, colsum, band, &sq, &bw, s, scratch);
            if (!rc) rc = form_phis(n2, J2, tau, 1, P2, colsum, band, &sq, &bw, s, scratch);
            if (rc) break;
            const double* M[2] = {P1[1], P2[1]};
            Epi e{};
            e.kind = EPI_EE; e.alpha = tau; e.U = U; e.status = p->status;
            double* outs[1] = {Y};
            rc = fp64_chain_m(p, M, X, outs, e, s);
            break;
        }
        case MM_LAWSON_EULER: {
            StencilArgs a = stencil_base(p, U, X, PRE_LAWSON, t, pg);
            a.ca = tau;
            rc = launch_prepass(a, s);
            if (rc) break;
            Epi e{};
            e.kind = EPI_STORE; e.alpha = 1.0; e.C = U;
            rc = run_tucker(p, 0, X, Y, e, s);
            break;
        }
        case MM_LAWSON2B: {
            StencilArgs a = stencil_base(p, U, X, PRE_LAWSON, t, pg);
            a.ca = tau; a.cb = 0.5 * tau; a.W2 = Z;
            rc = launch_prepass(a, s);
            if (rc) break;
            Epi e1{};
            e1.kind = EPI_STORE; e1.alpha = 1.0; e1.C = U2;
            rc = run_tucker(p, 0, X, Y, e1, s);
            if (rc) break;
            Epi e2{};
            e2.kind = EPI_LAWSON2; e2.alpha = 1.0; e2.beta = 0.5 * tau; e2.U = U; e2.U2 = U2;
            e2.t1 = t + tau; e2.g = pg; e2.status = p->status;
            rc = run_tucker(p, 0, Z, Y, e2, s);
            break;
        }
        default: rc = MM_ERR_ARG;
        }
    }
    return rc;
}

}  // namespace
