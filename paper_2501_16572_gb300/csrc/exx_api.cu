// C interface of libexx_gb300: argument checks, plan life cycle, and the host-side
// orchestration of the batched solve (Sec. II.B), the exchange accumulation (Eq. 1),
// the energy and the ACE construction (Sec. III.A).
#include "exx_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace exx {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    set_error(buf);
    return e == cudaErrorMemoryAllocation ? EXX_ERR_OOM : EXX_ERR_CUDA;
}

static int invalid(const char *msg)
{
    set_error(msg);
    return EXX_ERR_INVALID_ARG;
}

static std::atomic<uint64_t> g_epoch{0};
void bump_epoch(Plan &P) { P.epoch = ++g_epoch; }
static void graph_evict_plan(const Plan *P);

int dev_reserve(DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes && b.p) return EXX_OK;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) return EXX_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    b.bytes = bytes;
    return EXX_OK;
}

void dev_free(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

static void free_plan_buffers(Plan &P)
{
    for (auto &b : P.B64) dev_free(b);
    for (auto &row : P.Btc)
        for (auto &b : row) dev_free(b);
    for (auto &row : P.t3img)
        for (auto &b : row) dev_free(b);
    for (auto &row : P.t3imgc)
        for (auto &b : row) dev_free(b);
    dev_free(P.F32n);
    dev_free(P.orig_V);
    dev_free(P.F64n);
    dev_free(P.orig_ws);
    for (auto *b : {&P.cmats, &P.cFd, &P.cwork, &P.cpairs, &P.cred, &P.cace}) dev_free(*b);
    for (auto *b : {&P.F64, &P.F32, &P.work[0], &P.work[1], &P.work[2], &P.pairs_d, &P.blocks_d,
                    &P.acc_hi, &P.acc_lo, &P.g32, &P.psi32, &P.gemm_ws, &P.small_ws, &P.info_d,
                    &P.red_ws, &P.host_stage_psi, &P.host_stage_f, &P.host_stage_xi, &P.host_stage_w,
                    &P.err_d})
        dev_free(*b);
}

// Default batch size: enough fields per launch that every SM loops over tens of tiles
// (launch start-up and the last tile's drain are amortised), capped by a memory budget
// per batch buffer.
static int default_pairs(const Plan &P, int block)
{
    long per_field = long(P.N) * (P.prec == EXX_PREC_FP64 || P.prec == EXX_PREC_BF16X10 ? 8 : 4);
    long budget = 2048L << 20;   // per work buffer (two of them)
    long pairs = std::max<long>(block * block, budget / per_field);
    pairs = std::min<long>(pairs, 1024);
    return int((pairs / (block * block)) * (block * block));
}

static int ensure_schedule(Plan &P, int n_occ, int n_in, bool aliased, cudaStream_t s)
{
    const int block = P.block_orbitals > 0 ? P.block_orbitals : 8;
    const int maxp = P.pairs_per_batch > 0 ? P.pairs_per_batch : default_pairs(P, block);
    int key[4] = {n_occ, n_in, (aliased ? 1 : 0) | (block << 1), maxp};
    if (std::equal(key, key + 4, P.sched_key)) return EXX_OK;
    P.sched = build_schedule(n_occ, n_in, aliased, block, maxp);
    if (int rc = dev_reserve(P.pairs_d, std::max<size_t>(1, P.sched.pairs.size()) * sizeof(int2))) return rc;
    if (int rc = dev_reserve(P.blocks_d, std::max<size_t>(1, P.sched.blocks.size()) * sizeof(Block))) return rc;
    EXX_CUDA(cudaMemcpyAsync(P.pairs_d.p, P.sched.pairs.data(), P.sched.pairs.size() * sizeof(int2),
                             cudaMemcpyHostToDevice, s));
    EXX_CUDA(cudaMemcpyAsync(P.blocks_d.p, P.sched.blocks.data(), P.sched.blocks.size() * sizeof(Block),
                             cudaMemcpyHostToDevice, s));
    EXX_CUDA(cudaStreamSynchronize(s));   // host vectors may be rebuilt by the next call
    bump_epoch(P);
    std::copy(key, key + 4, P.sched_key);
    return EXX_OK;
}

int timing_begin(Plan &P, int kind, cudaStream_t s)
{
    if (!P.timing.on) return -1;
    TimingRec r{kind, nullptr, nullptr};
    for (cudaEvent_t *e : {&r.start, &r.stop}) {
        if (!P.timing.pool.empty()) {
            *e = P.timing.pool.back();
            P.timing.pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            return -1;
        }
    }
    cudaEventRecord(r.start, s);
    P.timing.recs.push_back(r);
    return int(P.timing.recs.size()) - 1;
}

void timing_end(Plan &P, int rec, cudaStream_t s)
{
    if (rec < 0 || rec >= int(P.timing.recs.size())) return;
    cudaEventRecord(P.timing.recs[rec].stop, s);
}

static void timing_recycle(Plan &P)
{
    for (auto &r : P.timing.recs) {
        P.timing.pool.push_back(r.start);
        P.timing.pool.push_back(r.stop);
    }
    P.timing.recs.clear();
}

}  // namespace exx

using namespace exx;

static Plan *as_plan(exx_plan p) { return reinterpret_cast<Plan *>(p); }

extern "C" {

const char *exx_status_string(int st)
{
    switch (st) {
    case EXX_OK: return "EXX_OK";
    case EXX_ERR_INVALID_ARG: return "EXX_ERR_INVALID_ARG: invalid argument";
    case EXX_ERR_CUDA: return "EXX_ERR_CUDA: CUDA call failed";
    case EXX_ERR_OOM: return "EXX_ERR_OOM: device allocation failed";
    case EXX_ERR_NOT_POSDEF: return "EXX_ERR_NOT_POSDEF: -M is not positive definite";
    case EXX_ERR_TIMEOUT: return "EXX_ERR_TIMEOUT: bounded device wait ran out";
    case EXX_ERR_UNSUPPORTED: return "EXX_ERR_UNSUPPORTED: unsupported combination";
    default: return "unknown exx status";
    }
}

const char *exx_last_error(void) { return g_last_error.c_str(); }

int exx_plan_create(exx_plan *out, int Nx, int Ny, int Nz, double h, const int bc[3], int fd_order,
                    int kernel, double omega)
{
    if (!out) return invalid("exx_plan_create: out is NULL");
    *out = nullptr;
    if (!bc) return invalid("exx_plan_create: bc is NULL");
    const int n[3] = {Nx, Ny, Nz};
    for (int d = 0; d < 3; ++d) {
        if (n[d] < 2 || n[d] > 256) return invalid("exx_plan_create: each grid size must be in [2, 256]");
        if (bc[d] != EXX_BC_DIRICHLET && bc[d] != EXX_BC_PERIODIC) return invalid("exx_plan_create: bad bc");
    }
    if (!(h > 0.0) || !std::isfinite(h)) return invalid("exx_plan_create: h must be > 0");
    if (fd_order < 2 || fd_order > 24 || (fd_order & 1)) return invalid("exx_plan_create: fd_order must be even in [2, 24]");
    if (kernel != EXX_KERNEL_COULOMB && kernel != EXX_KERNEL_ERFC && kernel != EXX_KERNEL_ERFC_PAPER16PI)
        return invalid("exx_plan_create: bad kernel");
    if (kernel != EXX_KERNEL_COULOMB && !(omega > 0.0)) return invalid("exx_plan_create: omega must be > 0 for a screened kernel");
    if (kernel == EXX_KERNEL_COULOMB && bc[0] == EXX_BC_PERIODIC && bc[1] == EXX_BC_PERIODIC &&
        bc[2] == EXX_BC_PERIODIC) {
        set_error("exx_plan_create: the unscreened kernel has a zero eigenvalue on an all-periodic grid");
        return EXX_ERR_UNSUPPORTED;
    }
    Plan *P = new Plan();
    for (int d = 0; d < 3; ++d) {
        P->n[d] = n[d];
        P->bc[d] = bc[d];
    }
    P->N = Nx * Ny * Nz;
    P->h = h;
    P->dV = h * h * h;
    P->omega = omega;
    P->fd_order = fd_order;
    P->kernel = kernel;
    // host FP64 setup, once per plan (Eqs. 6-7)
    for (int d = 0; d < 3; ++d) {
        int nd = n[d];
        std::vector<double> D(size_t(nd) * nd);
        second_derivative(nd, h, bc[d], fd_order / 2, D.data());
        P->V[d].resize(size_t(nd) * nd);
        P->lam[d].resize(nd);
        if (sym_eig(nd, D.data(), P->V[d].data(), P->lam[d].data())) {
            delete P;
            set_error("exx_plan_create: eigen-decomposition did not converge");
            return EXX_ERR_UNSUPPORTED;
        }
    }
    P->F.resize(size_t(P->N));
    for (int c = 0; c < Nz; ++c)
        for (int b = 0; b < Ny; ++b)
            for (int a = 0; a < Nx; ++a)
                P->F[a + size_t(Nx) * (b + size_t(Ny) * c)] =
                    kernel_f(P->lam[0][a] + P->lam[1][b] + P->lam[2][c], kernel, omega);
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "exx_plan_create: no usable CUDA device");
    }
    if (int rc = fp64_upload(*P)) {
        free_plan_buffers(*P);
        delete P;
        return rc;
    }
    bump_epoch(*P);
    *out = reinterpret_cast<exx_plan>(P);
    return EXX_OK;
}

int exx_plan_set_precision(exx_plan plan, int prec)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_plan_set_precision: plan is NULL");
    if (prec < EXX_PREC_FP64 || prec > EXX_PREC_BF16X7) return invalid("exx_plan_set_precision: bad precision");
    if (P->cplx && prec != EXX_PREC_FP64) {
        set_error("exx_plan_set_precision: Bloch plans run in FP64");
        return EXX_ERR_UNSUPPORTED;
    }
    if (prec == EXX_PREC_BF16X7) {
        if (int rc = tc3_upload(*P)) return rc;
    } else if (prec != EXX_PREC_FP64) {
        if (int rc = tc_upload(*P, prec)) return rc;
    }
    P->prec = prec;
    std::fill(P->sched_key, P->sched_key + 4, -1);
    bump_epoch(*P);
    return EXX_OK;
}

int exx_plan_set_batch(exx_plan plan, int pairs_per_batch, int block_orbitals)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_plan_set_batch: plan is NULL");
    if (pairs_per_batch < 0 || block_orbitals < 0 || block_orbitals > 32)
        return invalid("exx_plan_set_batch: sizes must be >= 0 (block <= 32)");
    P->pairs_per_batch = pairs_per_batch;
    P->block_orbitals = block_orbitals;
    std::fill(P->sched_key, P->sched_key + 4, -1);
    bump_epoch(*P);
    return EXX_OK;
}

int exx_plan_set_shard(exx_plan plan, int rank, int world)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_plan_set_shard: plan is NULL");
    if (world < 1 || rank < 0 || rank >= world) return invalid("exx_plan_set_shard: need 0 <= rank < world");
    P->shard_rank = rank;
    P->shard_world = world;
    bump_epoch(*P);
    return EXX_OK;
}

int exx_plan_destroy(exx_plan plan)
{
    Plan *P = as_plan(plan);
    if (!P) return EXX_OK;
    cudaDeviceSynchronize();
    graph_evict_plan(P);
    free_plan_buffers(*P);
    timing_recycle(*P);
    for (auto e : P->timing.pool) cudaEventDestroy(e);
    delete P;
    return EXX_OK;
}

int exx_plan_set_timing(exx_plan plan, int enable)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_plan_set_timing: plan is NULL");
    EXX_CUDA(cudaDeviceSynchronize());
    timing_recycle(*P);
    P->timing.on = enable != 0;
    return EXX_OK;
}

int exx_plan_get_timing(exx_plan plan, int kind, double *ms_h, long *launches_h)
{
    Plan *P = as_plan(plan);
    if (!P || !ms_h || !launches_h) return invalid("exx_plan_get_timing: NULL argument");
    if (kind < 0 || kind >= EXX_TIMING_KINDS) return invalid("exx_plan_get_timing: bad kind");
    EXX_CUDA(cudaDeviceSynchronize());
    double tot = 0.0;
    long cnt = 0;
    for (auto &r : P->timing.recs) {
        if (r.kind != kind) continue;
        float ms = 0.f;
        EXX_CUDA(cudaEventElapsedTime(&ms, r.start, r.stop));
        tot += ms;
        cnt++;
    }
    *ms_h = tot;
    *launches_h = cnt;
    return EXX_OK;
}

int exx_plan_get(exx_plan plan, int which, double *dst_h, long count)
{
    Plan *P = as_plan(plan);
    if (!P || !dst_h) return invalid("exx_plan_get: NULL argument");
    if (which >= 0 && which < 3) {
        if (count != P->n[which]) return invalid("exx_plan_get: count must equal n_d");
        std::copy(P->lam[which].begin(), P->lam[which].end(), dst_h);
        return EXX_OK;
    }
    if (which == 3) {
        if (count != P->N) return invalid("exx_plan_get: count must equal N");
        std::copy(P->F.begin(), P->F.end(), dst_h);
        return EXX_OK;
    }
    return invalid("exx_plan_get: which must be 0..3");
}

long exx_plan_launch_count(exx_plan plan)
{
    Plan *P = as_plan(plan);
    return P ? P->launches : -1;
}

}  // extern "C"

namespace exx {

struct ApplyCall {
    const double *Psi_occ; int n_occ; long ld_occ; const double *f;
    const double *Psi_in; int n_in; long ld_in; double *out; long ld_out;
    bool aliased;
};

// Checks, schedule and every device allocation of one exx_apply (synchronizes `s` when
// the schedule changes).  Nothing here is captured into a graph.
static int apply_prepare(Plan *P, ApplyCall &c, cudaStream_t s)
{
    if (!P) return invalid("exx_apply: plan is NULL");
    if (P->cplx) {
        set_error("exx_apply: a Bloch plan takes complex orbitals (exx_apply_complex)");
        return EXX_ERR_UNSUPPORTED;
    }
    if (!c.Psi_occ || !c.f || !c.Psi_in || !c.out) return invalid("exx_apply: NULL array");
    if (c.n_occ < 1 || c.n_in < 1 || c.n_occ > 65536 || c.n_in > 65536) return invalid("exx_apply: orbital counts must be in [1, 65536]");
    if (c.ld_occ < P->N || c.ld_in < P->N || c.ld_out < P->N) return invalid("exx_apply: leading dimensions must be >= N");
    const char *o0 = reinterpret_cast<const char *>(c.out);
    const char *o1 = o0 + (size_t(c.n_in - 1) * c.ld_out + P->N) * sizeof(double);
    auto overlaps = [&](const double *a, int n, long ld) {
        const char *a0 = reinterpret_cast<const char *>(a);
        const char *a1 = a0 + (size_t(n - 1) * ld + P->N) * sizeof(double);
        return a0 < o1 && o0 < a1;
    };
    if (overlaps(c.Psi_occ, c.n_occ, c.ld_occ) || overlaps(c.Psi_in, c.n_in, c.ld_in)) return invalid("exx_apply: out overlaps an input");
    c.aliased = (c.Psi_in == c.Psi_occ) && (c.ld_in == c.ld_occ) && (c.n_in >= c.n_occ);
    if (int rc = ensure_schedule(*P, c.n_occ, c.n_in, c.aliased, s)) return rc;
    const Schedule &S = P->sched;
    if (P->prec == EXX_PREC_FP64) {
        size_t fb = size_t(S.max_fields) * P->N * sizeof(double);
        if (int rc = dev_reserve(P->work[0], fb)) return rc;
        return dev_reserve(P->work[1], fb);
    }
    if (int rc = tc_reserve_orbitals(*P, c.n_occ, c.n_in, c.aliased)) return rc;
    const bool hl = tc_is_hilo(P->prec);
    P->tc_lo_off = hl ? long(S.max_fields) * P->N : 0;
    size_t fb = size_t(S.max_fields) * P->N * sizeof(float) * (hl ? 2 : 1);
    if (int rc = dev_reserve(P->work[0], fb)) return rc;
    return dev_reserve(P->work[1], fb);
}

// The launches of one exx_apply (stream work only: capturable into a CUDA graph).  With
// b_count >= 0 only batches [b_first, b_first + b_count) run (autotuner trials).
static int apply_launch(Plan *P, const ApplyCall &c, cudaStream_t s, int b_first = 0, int b_count = -1)
{
    const Schedule &S = P->sched;
    auto skip = [&](size_t b) {
        return b_count >= 0 && (int(b) < b_first || int(b) >= b_first + b_count);
    };
    const int2 *pairs_d = static_cast<const int2 *>(P->pairs_d.p);
    const Block *blocks_d = static_cast<const Block *>(P->blocks_d.p);
    if (P->prec == EXX_PREC_FP64) {
        EXX_CUDA(cudaMemset2DAsync(c.out, size_t(c.ld_out) * sizeof(double), 0, size_t(P->N) * sizeof(double),
                                   c.n_in, s));
        for (size_t b = 0; b < S.batches.size(); ++b) {
            if (int(b % P->shard_world) != P->shard_rank || skip(b)) continue;
            const Batch &bt = S.batches[b];
            double *V = nullptr;
            if (int rc = fp64_solve_batch(*P, c.Psi_occ, c.ld_occ, c.Psi_in, c.ld_in, pairs_d + S.pair0[b], bt.nfields,
                                          static_cast<double *>(P->work[0].p), static_cast<double *>(P->work[1].p), &V, s))
                return rc;
            if (int rc = fp64_accumulate(*P, c.Psi_occ, c.ld_occ, c.Psi_in, c.ld_in, c.f, blocks_d + bt.block0,
                                         bt.nblocks, V, c.out, c.ld_out, s))
                return rc;
        }
        return EXX_OK;
    }
    const int prec = P->prec;
    if (int rc = tc_prepare_orbitals(*P, c.Psi_occ, c.n_occ, c.ld_occ, c.f, c.Psi_in, c.n_in, c.ld_in, c.aliased, s))
        return rc;
    for (size_t b = 0; b < S.batches.size(); ++b) {
        if (int(b % P->shard_world) != P->shard_rank || skip(b)) continue;
        const Batch &bt = S.batches[b];
        if (int rc = tc_solve_batch(*P, prec, pairs_d + S.pair0[b], bt.nfields, static_cast<float *>(P->work[0].p),
                                    static_cast<float *>(P->work[1].p), s))
            return rc;
        if (int rc = tc_accumulate(*P, blocks_d + bt.block0, bt.nblocks, P->tc_result, s)) return rc;
    }
    return tc_finalize(*P, c.n_in, c.out, c.ld_out, s);
}

// Graphs of exx_apply_batched, keyed by everything the captured launches depend on.
struct GraphEntry {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
    std::vector<Plan *> plans;
    std::vector<long> launches;   // kernels each plan's part of the graph launches
};
static std::mutex g_graph_mutex;
static std::vector<GraphEntry> g_graphs;
constexpr size_t kMaxGraphs = 8;
constexpr int kBranches = 8;   // concurrent branches of a batched graph

// Drops every cached graph that launches work of plan P (called before P is freed).
static void graph_evict_plan(const Plan *P)
{
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    for (size_t i = 0; i < g_graphs.size();) {
        if (std::find(g_graphs[i].plans.begin(), g_graphs[i].plans.end(), P) != g_graphs[i].plans.end()) {
            cudaGraphExecDestroy(g_graphs[i].exec);
            g_graphs.erase(g_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

static void graph_key_add(std::vector<uintptr_t> &k, const Plan *P, const ApplyCall &c)
{
    const uintptr_t v[] = {uintptr_t(P), uintptr_t(P->epoch), uintptr_t(P->prec), uintptr_t(P->pairs_per_batch), uintptr_t(P->block_orbitals),
                           uintptr_t(P->shard_rank), uintptr_t(P->shard_world), uintptr_t(c.Psi_occ), uintptr_t(c.n_occ),
                           uintptr_t(c.ld_occ), uintptr_t(c.f), uintptr_t(c.Psi_in), uintptr_t(c.n_in), uintptr_t(c.ld_in),
                           uintptr_t(c.out), uintptr_t(c.ld_out), uintptr_t(P->work[0].p), uintptr_t(P->work[1].p),
                           uintptr_t(P->psi32.p), uintptr_t(P->g32.p), uintptr_t(P->acc_hi.p), uintptr_t(P->acc_lo.p),
                           uintptr_t(P->pairs_d.p), uintptr_t(P->blocks_d.p), uintptr_t(P->err_d.p),
                           uintptr_t(P->timing.on)};
    k.insert(k.end(), v, v + sizeof(v) / sizeof(v[0]));
}

}  // namespace exx

extern "C" {

int exx_apply(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
              const double *Psi_in, int n_in, long ld_in, double *out, long ld_out, exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    ApplyCall c{Psi_occ, n_occ, ld_occ, f, Psi_in, n_in, ld_in, out, ld_out, false};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = apply_prepare(P, c, s)) return rc;
    P->launches = 0;
    return apply_launch(P, c, s);
}

int exx_apply_original(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
                       const double *Psi_in, int n_in, long ld_in, double *out, long ld_out, exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_apply_original: plan is NULL");
    if (!Psi_occ || !f || !Psi_in || !out) return invalid("exx_apply_original: NULL array");
    if (n_occ < 1 || n_in < 1 || n_occ > 65536 || n_in > 65536)
        return invalid("exx_apply_original: orbital counts must be in [1, 65536]");
    if (ld_occ < P->N || ld_in < P->N || ld_out < P->N) return invalid("exx_apply_original: leading dimensions must be >= N");
    const char *o0 = reinterpret_cast<const char *>(out);
    const char *o1 = o0 + (size_t(n_in - 1) * ld_out + P->N) * sizeof(double);
    auto overlaps = [&](const double *a, int n, long ld) {
        const char *a0 = reinterpret_cast<const char *>(a);
        const char *a1 = a0 + (size_t(n - 1) * ld + P->N) * sizeof(double);
        return a0 < o1 && o0 < a1;
    };
    if (overlaps(Psi_occ, n_occ, ld_occ) || overlaps(Psi_in, n_in, ld_in)) return invalid("exx_apply_original: out overlaps an input");
    const bool aliased = (Psi_in == Psi_occ) && (ld_in == ld_occ) && (n_in >= n_occ);
    P->launches = 0;
    return original_apply(*P, Psi_occ, n_occ, ld_occ, f, Psi_in, n_in, ld_in, out, ld_out, aliased,
                          reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace exx {

// ---- autotuner: tile and schedule settings measured on the caller's grid and data ---------
struct TuneKey {
    int n[3], bc[3], prec, n_occ, n_in, aliased;
    bool operator==(const TuneKey &o) const
    {
        return std::equal(n, n + 3, o.n) && std::equal(bc, bc + 3, o.bc) && prec == o.prec && n_occ == o.n_occ &&
               n_in == o.n_in && aliased == o.aliased;
    }
};
struct TuneVal {
    int pairs, block, zwn, znbuf, stage, pipe;
    double ms;
};
static std::mutex g_tune_mutex;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

static void tune_set(Plan &P, const TuneVal &v)
{
    P.pairs_per_batch = v.pairs;
    P.block_orbitals = v.block;
    P.t3_zwn = v.zwn;
    P.t3_znbuf = v.znbuf;
    P.t3_stage = v.stage;
    P.t3_pipe = v.pipe;
    std::fill(P.sched_key, P.sched_key + 4, -1);
    bump_epoch(P);
}

// Device time per pair solve of batches [b0, b0 + nb) with setting v (one warm-up run, then
// one timed run, CUDA events on s); +inf when the setting does not apply.
static double tune_trial(Plan &P, ApplyCall c, const TuneVal &v, cudaStream_t s, int &rc)
{
    rc = EXX_OK;
    tune_set(P, v);
    if (P.prec == EXX_PREC_BF16X7 && (rc = tc3_upload(P)) != EXX_OK) return 1e300;
    if ((rc = apply_prepare(&P, c, s)) != EXX_OK) return 1e300;
    const int nb = int(P.sched.batches.size());
    const int b0 = nb > 2 ? 1 : 0, cnt = std::min(3, nb - b0);
    long pairs = 0;
    for (int b = b0; b < b0 + cnt; ++b) pairs += P.sched.batches[b].nfields;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = EXX_ERR_CUDA;
        return 1e300;
    }
    double ms = 1e300;
    if ((rc = apply_launch(&P, c, s, b0, cnt)) == EXX_OK) {
        cudaEventRecord(e0, s);
        rc = apply_launch(&P, c, s, b0, cnt);
        cudaEventRecord(e1, s);
        float t = 0.f;
        if (rc == EXX_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            ms = double(t) / double(std::max(1L, pairs));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace exx

extern "C" {

int exx_plan_autotune(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
                      const double *Psi_in, int n_in, long ld_in, double *out, long ld_out, int flags,
                      exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    ApplyCall c{Psi_occ, n_occ, ld_occ, f, Psi_in, n_in, ld_in, out, ld_out, false};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = apply_prepare(P, c, s)) return rc;   // argument checks, aliasing
    TuneKey key{{P->n[0], P->n[1], P->n[2]}, {P->bc[0], P->bc[1], P->bc[2]}, P->prec, n_occ, n_in, c.aliased ? 1 : 0};
    if (!(flags & 1)) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (auto &kv : g_tune_cache)
            if (kv.first == key) {
                tune_set(*P, kv.second);
                if (P->prec == EXX_PREC_BF16X7)
                    if (int rc = tc3_upload(*P)) return rc;
                P->tuned = 2;
                P->tune_ms = kv.second.ms;
                return EXX_OK;
            }
    }
    // coordinate descent: pair batch and orbital block, then (three-pass mode) the pass-B
    // matrix blocks and buffers, then the slice-pass staging
    TuneVal best{0, 0, 0, 0, -1, -1, 1e300};
    auto consider = [&](TuneVal v) -> int {
        int rc = EXX_OK;
        v.ms = tune_trial(*P, c, v, s, rc);
        if (rc != EXX_OK && rc != EXX_ERR_UNSUPPORTED && rc != EXX_ERR_OOM) return rc;
        if (rc == EXX_OK && v.ms < best.ms) best = v;
        return EXX_OK;
    };
    for (int pairs : {0, 256, 512, 1024})
        for (int block : {8, 16})
            if (int rc = consider({pairs, block, 0, 0, -1, -1, 0.0})) return rc;
    if (P->prec == EXX_PREC_BF16X7) {
        const TuneVal base = best;
        for (auto &zc : tc3_z_choices(P->n[2]))
            if (int rc = consider({base.pairs, base.block, zc.first, zc.second, -1, -1, 0.0})) return rc;
        const TuneVal base2 = best;
        for (int pipe : {0, 1})
            for (int st : {-1, 0, 1})
                if (int rc = consider({base2.pairs, base2.block, base2.zwn, base2.znbuf, st, pipe, 0.0})) return rc;
    }
    if (best.ms >= 1e300) {
        set_error("exx_plan_autotune: no candidate setting ran");
        return EXX_ERR_UNSUPPORTED;
    }
    tune_set(*P, best);
    if (P->prec == EXX_PREC_BF16X7)
        if (int rc = tc3_upload(*P)) return rc;
    if (int rc = apply_prepare(P, c, s)) return rc;
    P->tuned = 1;
    P->tune_ms = best.ms;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (auto &kv : g_tune_cache)
        if (kv.first == key) {
            kv.second = best;
            return EXX_OK;
        }
    g_tune_cache.push_back({key, best});
    return EXX_OK;
}

int exx_plan_set_tuning(exx_plan plan, const int *settings_h)
{
    Plan *P = as_plan(plan);
    if (!P || !settings_h) return invalid("exx_plan_set_tuning: NULL argument");
    const int *v = settings_h;
    if (v[0] < 0 || v[1] < 0 || v[1] > 32 || v[2] < -256 || v[2] > 256 || (std::abs(v[2]) & 15) || v[3] < 0 || v[3] > 64 ||
        v[4] < -1 || v[4] > 1 || v[5] < -1 || v[5] > 1 || ((v[2] == 0) != (v[3] == 0)))
        return invalid("exx_plan_set_tuning: settings out of range");
    tune_set(*P, {v[0], v[1], v[2], v[3], v[4], v[5], 0.0});
    if (P->prec == EXX_PREC_BF16X7)
        if (int rc = tc3_upload(*P)) return rc;
    P->tuned = 0;
    P->tune_ms = 0.0;
    return EXX_OK;
}

int exx_plan_get_tuning(exx_plan plan, int *settings_h, double *ms_per_pair_h, int *tuned_h)
{
    Plan *P = as_plan(plan);
    if (!P || !settings_h || !ms_per_pair_h || !tuned_h) return invalid("exx_plan_get_tuning: NULL argument");
    settings_h[0] = P->pairs_per_batch;
    settings_h[1] = P->block_orbitals;
    settings_h[2] = P->t3_zwn;
    settings_h[3] = P->t3_znbuf;
    settings_h[4] = P->t3_stage;
    settings_h[5] = P->t3_pipe;
    *ms_per_pair_h = P->tune_ms;
    *tuned_h = P->tuned;
    return EXX_OK;
}

int exx_energy(exx_plan plan, const double *Psi_occ, int n_occ, long ld, const double *f, const double *VxPsi,
               long ld_v, double *E_x_h, exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_energy: plan is NULL");
    if (!Psi_occ || !f || !VxPsi || !E_x_h) return invalid("exx_energy: NULL argument");
    if (n_occ < 1 || ld < P->N || ld_v < P->N) return invalid("exx_energy: bad sizes");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = tc_check_error(*P, s)) return rc;   // a bounded wait of an earlier exx_apply ran out
    P->launches = 0;
    return energy_fp64(*P, Psi_occ, n_occ, ld, f, VxPsi, ld_v, E_x_h, s);
}

int ace_build(exx_plan plan, const double *Psi, int n, long ld, const double *W, long ld_w, double *xi,
              long ld_xi, double *M_out, int *info_h, exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("ace_build: plan is NULL");
    if (!Psi || !W || !xi || !info_h) return invalid("ace_build: NULL argument");
    if (n < 1 || n > 2048 || ld < P->N || ld_w < P->N || ld_xi < P->N) return invalid("ace_build: bad sizes");
    *info_h = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (int rc = tc_check_error(*P, s)) return rc;
    P->launches = 0;
    // device scratch: M (n x n), Linv (n x n), info
    size_t nn = size_t(n) * n;
    if (int rc = dev_reserve(P->info_d, 2 * nn * sizeof(double) + 256)) return rc;
    double *M = M_out ? M_out : static_cast<double *>(P->info_d.p);
    double *Linv = static_cast<double *>(P->info_d.p) + nn;
    int *info_d = reinterpret_cast<int *>(static_cast<double *>(P->info_d.p) + 2 * nn);
    // split-precision plans take the ACE products on the tensor cores, FP64 plans on the
    // CUDA cores; the Cholesky factor and its inverse are FP64 in both
    const bool tcg = P->prec != EXX_PREC_FP64;
    if (tcg) {
        if (int rc = tc_gemm(*P, n, n, P->N, Psi, ld, 1, W, ld_w, 1, P->dV, M, 1, n, s)) return rc;
    } else if (int rc = gemm_fp64_tn_splitk(*P, n, n, P->N, Psi, ld, W, ld_w, P->dV, M, n, s)) {
        return rc;
    }
    if (int rc = cholesky_neg_sym_and_inverse(*P, n, M, Linv, info_d, s)) return rc;
    int info = 0;
    EXX_CUDA(cudaMemcpyAsync(&info, info_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaStreamSynchronize(s));
    if (info) {
        *info_h = info;
        set_error("ace_build: -sym(M) is not positive definite");
        return EXX_ERR_NOT_POSDEF;
    }
    // xi = W Linv^T
    if (tcg) {
        if (int rc = tc_gemm(*P, P->N, n, n, W, 1, ld_w, Linv, 1, n, 1.0, xi, 1, ld_xi, s)) return rc;
    } else if (int rc = gemm_fp64_nt(*P, P->N, n, n, W, ld_w, Linv, n, 1.0, xi, ld_xi, s)) {
        return rc;
    }
    EXX_CUDA(cudaStreamSynchronize(s));
    if (tcg) return tc_check_error(*P, s);
    return EXX_OK;
}

int ace_apply(exx_plan plan, const double *xi, int n, long ld_xi, const double *Phi, int nphi, long ld_phi,
              double *out, long ld_out, exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("ace_apply: plan is NULL");
    if (!xi || !Phi || !out) return invalid("ace_apply: NULL argument");
    if (n < 1 || nphi < 1 || n > 65536 || ld_xi < P->N || ld_phi < P->N || ld_out < P->N) return invalid("ace_apply: bad sizes");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    P->launches = 0;
    size_t need = size_t(n) * nphi * sizeof(double);
    if (int rc = dev_reserve(P->small_ws, need)) return rc;
    double *chi = static_cast<double *>(P->small_ws.p);
    // chi = xi^T Phi (n x nphi), out = -dV xi chi
    if (P->prec != EXX_PREC_FP64) {   // the two products on the tensor cores
        if (int rc = tc_gemm(*P, n, nphi, P->N, xi, ld_xi, 1, Phi, ld_phi, 1, 1.0, chi, 1, n, s)) return rc;
        return tc_gemm(*P, P->N, nphi, n, xi, 1, ld_xi, chi, n, 1, -P->dV, out, 1, ld_out, s);
    }
    if (int rc = gemm_fp64_tn_splitk(*P, n, nphi, P->N, xi, ld_xi, Phi, ld_phi, 1.0, chi, n, s)) return rc;
    return gemm_fp64_nn(*P, P->N, nphi, n, xi, ld_xi, chi, n, -P->dV, out, ld_out, s);
}

int exx_ace_step_host(exx_plan plan, const double *Psi_h, int n, long ld, int n_occ, const double *f_h,
                      double *xi_h, long ld_xi, double *E_x_h, int *info_h, exx_stream_t stream)
{
    Plan *P = as_plan(plan);
    if (!P) return invalid("exx_ace_step_host: plan is NULL");
    if (!Psi_h || !f_h || !xi_h || !E_x_h || !info_h) return invalid("exx_ace_step_host: NULL argument");
    if (n < 1 || n_occ < 1 || n_occ > n || ld < P->N || ld_xi < P->N) return invalid("exx_ace_step_host: bad sizes");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t cols = size_t(P->N) * n * sizeof(double);
    if (int rc = dev_reserve(P->host_stage_psi, cols)) return rc;
    if (int rc = dev_reserve(P->host_stage_w, cols)) return rc;
    if (int rc = dev_reserve(P->host_stage_xi, cols)) return rc;
    if (int rc = dev_reserve(P->host_stage_f, size_t(n_occ) * sizeof(double))) return rc;
    double *Psi = static_cast<double *>(P->host_stage_psi.p);
    double *W = static_cast<double *>(P->host_stage_w.p);
    double *xi = static_cast<double *>(P->host_stage_xi.p);
    double *f = static_cast<double *>(P->host_stage_f.p);
    // one contiguous copy when the host columns are packed (a pitched copy moves row by row
    // and runs far below the host link's bandwidth)
    if (ld == P->N)
        EXX_CUDA(cudaMemcpyAsync(Psi, Psi_h, cols, cudaMemcpyHostToDevice, s));
    else
        EXX_CUDA(cudaMemcpy2DAsync(Psi, size_t(P->N) * sizeof(double), Psi_h, size_t(ld) * sizeof(double),
                                   size_t(P->N) * sizeof(double), n, cudaMemcpyHostToDevice, s));
    EXX_CUDA(cudaMemcpyAsync(f, f_h, size_t(n_occ) * sizeof(double), cudaMemcpyHostToDevice, s));
    long launches = 0;
    if (int rc = exx_apply(plan, Psi, n_occ, P->N, f, Psi, n, P->N, W, P->N, stream)) return rc;
    launches += P->launches;
    if (int rc = exx_energy(plan, Psi, n_occ, P->N, f, W, P->N, E_x_h, stream)) return rc;
    launches += P->launches;
    int rc = ace_build(plan, Psi, n, P->N, W, P->N, xi, P->N, nullptr, info_h, stream);
    launches += P->launches;
    P->launches = launches;
    if (rc) return rc;
    if (ld_xi == P->N)
        EXX_CUDA(cudaMemcpyAsync(xi_h, xi, cols, cudaMemcpyDeviceToHost, s));
    else
        EXX_CUDA(cudaMemcpy2DAsync(xi_h, size_t(ld_xi) * sizeof(double), xi, size_t(P->N) * sizeof(double),
                                   size_t(P->N) * sizeof(double), n, cudaMemcpyDeviceToHost, s));
    EXX_CUDA(cudaStreamSynchronize(s));
    return EXX_OK;
}

int exx_apply_batched(const exx_plan *plans, int nsys, const exx_apply_args *args, exx_stream_t stream)
{
    if (!plans || !args || nsys < 1) return invalid("exx_apply_batched: bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<ApplyCall> calls(nsys);
    std::vector<uintptr_t> key;
    int prec0 = -1;
    // a plan holds one pair schedule and one workspace: the same plan twice in one call
    // would run the earlier system with the later system's schedule
    for (int i = 0; i < nsys; ++i)
        for (int j = 0; j < i; ++j)
            if (plans[i] == plans[j]) return invalid("exx_apply_batched: a plan appears more than once in plans[]");
    for (int i = 0; i < nsys; ++i) {
        Plan *P = as_plan(plans[i]);
        if (!P) return invalid("exx_apply_batched: NULL plan");
        if (prec0 < 0) prec0 = P->prec;
        if (P->prec != prec0) return invalid("exx_apply_batched: every plan must use the same precision");
        calls[i] = ApplyCall{args[i].Psi_occ, args[i].n_occ, args[i].ld_occ, args[i].f, args[i].Psi_in,
                             args[i].n_in, args[i].ld_in, args[i].out, args[i].ld_out, false};
        if (int rc = apply_prepare(P, calls[i], s)) return rc;   // all allocation happens here
    }
    for (int i = 0; i < nsys; ++i) graph_key_add(key, as_plan(plans[i]), calls[i]);
    bool any_timing = false;
    for (int i = 0; i < nsys; ++i) any_timing |= as_plan(plans[i])->timing.on;
    if (s == nullptr || any_timing) {   // legacy stream or per-launch timing: no graph
        for (int i = 0; i < nsys; ++i) as_plan(plans[i])->launches = 0;
        for (int i = 0; i < nsys; ++i)
            if (int rc = apply_launch(as_plan(plans[i]), calls[i], s)) return rc;
        return EXX_OK;
    }
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    for (auto &g : g_graphs)
        if (g.key == key) {
            EXX_CUDA(cudaGraphLaunch(g.exec, s));
            for (int i = 0; i < nsys; ++i) g.plans[i]->launches = 0;
            for (int i = 0; i < nsys; ++i) g.plans[i]->launches += g.launches[i];
            return EXX_OK;
        }
    // first call with this key: capture every system's launches into one graph
    GraphEntry ent;
    ent.key = key;
    for (int i = 0; i < nsys; ++i) {
        ent.plans.push_back(as_plan(plans[i]));
        ent.plans.back()->launches = 0;
    }
    // the systems' launch sequences go to kBranches forked streams inside the capture, so
    // the graph holds independent branches: small systems run concurrently and fill the
    // SMs that one system alone leaves idle
    const int nbr = std::min(nsys, kBranches);
    std::vector<cudaStream_t> side(nbr, nullptr);
    std::vector<cudaEvent_t> joins(nbr, nullptr);
    cudaEvent_t fork = nullptr;
    for (int k = 0; k < nbr; ++k) {
        EXX_CUDA(cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking));
        EXX_CUDA(cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming));
    }
    EXX_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    auto cleanup = [&]() {
        for (int k = 0; k < nbr; ++k) {
            cudaStreamDestroy(side[k]);
            cudaEventDestroy(joins[k]);
        }
        cudaEventDestroy(fork);
    };
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "exx_apply_batched: cudaStreamBeginCapture");
    }
    int rc = EXX_OK;
    if (cudaEventRecord(fork, s) != cudaSuccess) rc = EXX_ERR_CUDA;
    for (int k = 0; k < nbr && rc == EXX_OK; ++k)
        if (cudaStreamWaitEvent(side[k], fork, 0) != cudaSuccess) rc = EXX_ERR_CUDA;
    for (int i = 0; i < nsys && rc == EXX_OK; ++i) {
        const long before = ent.plans[i]->launches;
        rc = apply_launch(ent.plans[i], calls[i], side[i % nbr]);
        ent.launches.push_back(ent.plans[i]->launches - before);
    }
    for (int k = 0; k < nbr; ++k) {   // join every branch back, also after an error
        cudaEventRecord(joins[k], side[k]);
        cudaStreamWaitEvent(s, joins[k], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    cleanup();
    if (rc != EXX_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "exx_apply_batched: cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ent.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "exx_apply_batched: cudaGraphInstantiate");
    if (g_graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(ent);
    EXX_CUDA(cudaGraphLaunch(ent.exec, s));
    return EXX_OK;
}

}  // extern "C"
