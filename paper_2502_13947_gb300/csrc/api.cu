// api.cu -- the extern "C" entry points of libicd2s.so (declared in
// include/icd2s.h): argument checks, device memory owned by the handles,
// host tables, and the orchestration of one outer iteration of Algorithm 2
// as a fixed sequence of kernel launches on the caller's stream.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/icd2s.h"
#include "common.cuh"

using namespace icd2s;

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void icd2s::note_launch(int kernels) { g_launches.fetch_add((unsigned long long)kernels, std::memory_order_relaxed); }

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? ICD2S_ERR_OOM : ICD2S_ERR_CUDA,          \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define REQ(cond, code, ...)                \
    do {                                    \
        if (!(cond)) return fail(code, __VA_ARGS__); \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

void icd2s::set_error_message(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

namespace {

// Host tables.  The cosine temperature schedule of the emulated Ising
// machine, BETA[k] = round(2^24 / T_k) with
// T_k = T_min + (T_max - T_min)(1 + cos(pi k / (K - 1))) / 2 (T_0 = T_min when
// K = 1), and NLOG[j] = round(2^24 (-ln((j + 0.5) / 4096))): the test
// l * BETA[k] < NLOG[u >> 20] accepts a move of gain l > 0 with the
// Metropolis probability exp(-l / T_k) quantised to 1/4096.  Built with
// -ffp-contract=off so the doubles round identically on every host.
void make_beta(int sweeps, double T_max, double T_min, uint32_t* beta)
{
    for (int k = 0; k < sweeps; ++k) {
        double T;
        if (sweeps > 1)
            T = T_min + (T_max - T_min) * (1.0 + std::cos(M_PI * (double)k / (double)(sweeps - 1))) / 2.0;
        else
            T = T_min;
        const double b = 16777216.0 / T;
        beta[k] = (b < 4294967295.0) ? (uint32_t)std::llround(b) : 4294967295u;
    }
}

void make_nlog(uint32_t* nlog)
{
    for (int j = 0; j < 4096; ++j) nlog[j] = (uint32_t)std::llround(16777216.0 * -std::log(((double)j + 0.5) / 4096.0));
}

// Mutation rate of the MRAnnealer, Eq. 5: r_t = 0.3 (1 + cos(pi t / 15)) 0.99^t.
double mutation_rate(int t) { return 0.3 * (1.0 + std::cos(M_PI * (double)t / 15.0)) * std::pow(0.99, (double)t); }

// Allocations that may still succeed before the forced-failure hook makes the
// rest fail (icd2s_debug_fail_allocations_after; < 0: off).
std::atomic<long long> g_alloc_left{-1};

// Every device allocation of the library.  A failed one leaves *p null and no
// pending runtime error (which a later launch check would otherwise report).
cudaError_t dmalloc(void** p, size_t bytes)
{
    *p = nullptr;
    for (long long left = g_alloc_left.load(); left >= 0; left = g_alloc_left.load()) {
        if (left == 0) return cudaErrorMemoryAllocation;
        if (g_alloc_left.compare_exchange_weak(left, left - 1)) break;
    }
    const cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
    }
    return e;
}

template <class T>
cudaError_t dalloc(T** p, size_t count)
{
    void* v = nullptr;
    const cudaError_t e = dmalloc(&v, (count ? count : 1) * sizeof(T));
    *p = static_cast<T*>(v);
    return e;
}

// Frees every non-null pointer of a group and nulls it.
template <class... T>
void free_group(T**... p) { ((*p ? (void)cudaFree(*p) : (void)0, *p = nullptr), ...); }

}  // namespace

struct icd2s_qubo {
    int n = 0, ld = 0;
    int8_t* Q = nullptr;
    int32_t* diag = nullptr;
    int32_t* eta = nullptr;
    int32_t* etahat = nullptr;
    long long gain_bound = 0;  // max over j and x of |g_j|: bounds every gain of every solution (attained)
    int8_t* Q2 = nullptr;      // signed row pairs for the Tabu search (made when a state asks for them)
    bool has_m128 = false;     // an entry is -128: no signed rows (its negation is not an int8)
    // Q on parity labels (even Q_jj first), made at creation when the gain bound
    // is too wide for the compact Tabu keys on indices but fits them on labels
    int8_t* Qpk = nullptr;
    int32_t* pk_perm = nullptr;
    int pk_n0 = 0;
    // scratch of icd2s_energy (grown on demand)
    int cap = 0;
    uint8_t* xpad = nullptr;
    int32_t* hpad = nullptr;
    void* Qb = nullptr;  // bf16 copy of Q for the tensor-core refresh (made on first use)
};

// Proposal network: float32 master weights with Adam moments, the BF16 copy
// the kernels compute with, and the training scratch.
struct icd2s_mlp {
    uint64_t seed = 0;
    float* master = nullptr; float* mom = nullptr; float* vel = nullptr;
    void* Wb = nullptr;                       // bf16 [kNPar]
    float* partial = nullptr; size_t partial_cap = 0;
    float* losses = nullptr; int loss_cap = 0;
    int64_t adam_t = 0;                       // Adam steps taken
    bool tensor_cores = false;                // gradient contractions on the tensor cores (BF16 activations)
};

struct icd2s_state {
    icd2s_qubo* q = nullptr;
    int R = 0;
    uint64_t seed = 0;
    Dev d{};
    // device buffers owned by the state (Dev holds the same pointers)
    uint8_t* X = nullptr; int32_t* G = nullptr; int64_t* E = nullptr;
    int32_t* T = nullptr; int32_t* C = nullptr;
    int32_t* gamma = nullptr; int32_t* A = nullptr; int32_t* delta = nullptr; int32_t* order = nullptr;
    uint8_t* sel = nullptr;
    int32_t* FL = nullptr; int32_t* FCNT = nullptr; unsigned long long* DEACC = nullptr; unsigned int* DONE = nullptr;
    uint8_t* best_x = nullptr; int64_t* best_E = nullptr; int32_t* flags = nullptr;
    int32_t* idx = nullptr; int32_t* off = nullptr;
    uint8_t* scratch = nullptr;  // [R][ld] bytes: masks, unpadded host staging
    int64_t* counters = nullptr; // [0] anneal attempts
    uint32_t* nlog = nullptr;
    uint32_t* beta = nullptr; int beta_cap = 0;
    int* limtab = nullptr;  // [beta_cap][4096] acceptance limits of the schedule
    int beta_sweeps = -1; double beta_tmax = 0, beta_tmin = 0;
    bool have_select = false; int sel_K = 0;
    icd2s_tuning tune{-1, 0, 0, 0, {0}};  // kernel variants (see icd2s_set_tuning)
    // persistent anneal queue (uneven subQUBOs) and the iteration context of a captured step
    int32_t* lpt = nullptr;      // [R * 64] subQUBOs in largest-first order
    int32_t* queue = nullptr;    // [1] queue counter
    int32_t* ctx = nullptr;      // [4] ctx[0] = iteration number read by a replayed step
    double* rates = nullptr; int rates_cap = 0; int rates_mode = -1; double rates_const = 0;
    unsigned gen = 0;            // bumped whenever a buffer or a launch configuration changes
    cudaGraphExec_t graph = nullptr;
    icd2s_params graph_p{};
    unsigned graph_gen = 0;
    int dev_t = -1;              // value of ctx[0] after the last replay (-1: unknown)
    cudaStream_t own_stream = nullptr;  // captures cannot use the legacy default stream
    cudaEvent_t join_ev = nullptr;
    // dense refresh buffers (made on first use)
    void* Xb = nullptr; int32_t* G2 = nullptr; int64_t* E2 = nullptr; int* rflags = nullptr;  // [0] timeout, [1] mismatches
    cudaEvent_t rev[2] = {};  // around the tensor-core kernel of the last refresh (when timing)
    bool timed_refresh = false;
    int refresh_stall = 0;                          // fault injection: refreshes left whose loads are skipped
    unsigned long long refresh_stall_wait_ns = 0;   // and their wait bound
    cudaEvent_t aev[2] = {};  // around the write-back kernel of the last apply_flips_update_gains
    bool timed_apply = false;
    // phase timing of icd2s_step: events [2 * phase] / [2 * phase + 1]
    bool timing = false, timed_step = false;
    cudaEvent_t ev[2 * ICD2S_PHASES] = {};
    nvtxRangeId_t nvtx[ICD2S_PHASES] = {};  // the open NVTX range of each phase
    unsigned long long graph_kernels = 0;  // kernels in one replay of the captured step
    // learned selection
    int32_t* H = nullptr;                    // [R][ld] hit counts
    int32_t* ACC = nullptr; unsigned* TT = nullptr;  // split write-back: partial-sum planes, tile tickets
    float* F = nullptr; float* score = nullptr; int32_t* gmax = nullptr;  // made on first use
    uint16_t* tlog = nullptr; long long tlog_cap = 0;  // Tabu move logs beyond shared memory (on first use)
    bool have_features = false, have_scores = false;
    icd2s_mlp* mlp = nullptr;                // borrowed
    // improvement log (ring buffer)
    int log_cap = 0;
    float* LF = nullptr; uint8_t* LY = nullptr; int32_t* lrep = nullptr; uint8_t* prev_x = nullptr;
    int32_t* log_ctl = nullptr;              // {entries, capacity}
};

// Opens (which == 0) or closes (which == 1) a phase of icd2s_step: an NVTX
// range named for it (host side; a profiler can filter kernels by it) and,
// when timing, a CUDA event on the stream.
static void mark(icd2s_state* st, int phase, int which, cudaStream_t s)
{
    static const char* const kPhaseName[ICD2S_PHASES] = {
        "icd2s.tabu", "icd2s.select", "icd2s.anneal", "icd2s.apply_anneal", "icd2s.mutate", "icd2s.apply_mutate",
        "icd2s.best"};
    // start/end ranges (not a push/pop stack): a step that fails between the two
    // leaves one range open instead of unbalancing every later one
    if (which == 0) st->nvtx[phase] = nvtxRangeStartA(kPhaseName[phase]);
    else nvtxRangeEnd(st->nvtx[phase]);
    if (st->timing) cudaEventRecord(st->ev[2 * phase + which], s);
}

static void free_state(icd2s_state* st)
{
    void* ptrs[] = {st->X, st->G, st->E, st->T, st->C, st->gamma, st->A, st->delta, st->order, st->sel,
                    st->FL, st->FCNT, st->DEACC, st->DONE, st->best_x, st->best_E, st->flags, st->idx,
                    st->off, st->scratch, st->counters, st->nlog, st->beta, st->limtab,
                    st->lpt, st->queue, st->ctx, st->rates, st->Xb, st->G2, st->E2, st->rflags,
                    st->H, st->F, st->score, st->gmax, st->LF, st->LY, st->lrep, st->prev_x, st->log_ctl,
                    st->ACC, st->TT, st->tlog};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (st->graph) cudaGraphExecDestroy(st->graph);
    if (st->own_stream) cudaStreamDestroy(st->own_stream);
    if (st->join_ev) cudaEventDestroy(st->join_ev);
    for (cudaEvent_t e : st->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : st->rev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : st->aev)
        if (e) cudaEventDestroy(e);
    delete st;
}

// Mutation rates r_0 .. r_{upto-1} in device memory, for replayed steps.
static int ensure_rates(icd2s_state* st, int mut_mode, double mut_rate, int upto, cudaStream_t s)
{
    if (mut_mode == st->rates_mode && (mut_mode == 1 ? mut_rate == st->rates_const : true) && upto <= st->rates_cap)
        return ICD2S_OK;
    int cap = st->rates_cap > 0 ? st->rates_cap : 1024;
    while (cap < upto) cap *= 2;
    std::vector<double> r((size_t)cap);
    for (int t = 0; t < cap; ++t) r[t] = mut_mode == 0 ? mutation_rate(t) : mut_rate;
    CK(cudaStreamSynchronize(s));
    if (cap > st->rates_cap) {
        if (st->rates) CK(cudaFree(st->rates));
        st->rates = nullptr;
        st->rates_cap = 0;
        ++st->gen;
        CK(dalloc(&st->rates, (size_t)cap));
        st->rates_cap = cap;
    }
    CK(cudaMemcpy(st->rates, r.data(), sizeof(double) * cap, cudaMemcpyHostToDevice));
    st->rates_mode = mut_mode;
    st->rates_const = mut_rate;
    return ICD2S_OK;
}

static int ensure_beta(icd2s_state* st, int sweeps, double T_max, double T_min, cudaStream_t s)
{
    if (sweeps == st->beta_sweeps && T_max == st->beta_tmax && T_min == st->beta_tmin) return ICD2S_OK;
    REQ(sweeps >= 1 && sweeps <= kMaxSweeps, ICD2S_ERR_RANGE, "sweeps=%d outside 1..%d", sweeps, kMaxSweeps);
    if (sweeps > st->beta_cap) {
        CK(cudaStreamSynchronize(s));
        if (st->beta) CK(cudaFree(st->beta));
        if (st->limtab) CK(cudaFree(st->limtab));
        ++st->gen;  // a captured step holds the old pointers
        st->beta = nullptr;
        st->limtab = nullptr;
        st->beta_cap = 0;
        CK(dalloc(&st->beta, (size_t)sweeps));
        CK(dalloc(&st->limtab, (size_t)sweeps * 4096));
        st->beta_cap = sweeps;
    }
    std::vector<uint32_t> b((size_t)sweeps);
    make_beta(sweeps, T_max, T_min, b.data());
    CK(cudaMemcpyAsync(st->beta, b.data(), sizeof(uint32_t) * sweeps, cudaMemcpyHostToDevice, s));
    CK(launch_limtab(st->beta, sweeps, st->nlog, st->limtab, s));
    CK(cudaStreamSynchronize(s));  // the host vector dies here
    st->beta_sweeps = sweeps; st->beta_tmax = T_max; st->beta_tmin = T_min;
    return ICD2S_OK;
}

static int check_params(const icd2s_state* st, const icd2s_params* p)
{
    const int n = st->q->n;
    REQ(p, ICD2S_ERR_ARG, "params is NULL");
    REQ(p->z == st->d.z_total, ICD2S_ERR_ARG, "params z=%d differs from the state's replica set of %d", p->z,
        st->d.z_total);
    REQ(p->K >= 1 && p->K <= 64, ICD2S_ERR_RANGE, "K=%d outside 1..64", p->K);
    REQ(p->m_min >= 1 && p->m_min <= p->m_max && p->m_max <= kMaxM, ICD2S_ERR_RANGE,
        "subQUBO sizes m_min=%d m_max=%d outside 1..256", p->m_min, p->m_max);
    REQ((long long)p->K * p->m_max <= n, ICD2S_ERR_ARG, "K*m_max=%lld exceeds n=%d", (long long)p->K * p->m_max, n);
    const int mi = p->m_init > 0 ? p->m_init : p->m_max;
    REQ(mi <= kMaxM && mi <= n, ICD2S_ERR_RANGE, "m_init=%d outside 1..min(256, n)", mi);
    REQ(p->alpha >= 0, ICD2S_ERR_ARG, "alpha < 0");
    REQ(p->c >= 1 && p->c <= n, ICD2S_ERR_ARG, "tenure c=%d outside 1..n", p->c);
    REQ(p->sweeps >= 1 && p->sweeps <= kMaxSweeps, ICD2S_ERR_RANGE, "sweeps=%d outside 1..%d", p->sweeps,
        kMaxSweeps);
    REQ(p->T_min > 0 && p->T_max >= p->T_min, ICD2S_ERR_ARG, "need 0 < T_min <= T_max");
    const int64_t wl = (int64_t)1 << 24;
    REQ(p->w1 >= -wl && p->w1 <= wl && p->w2 >= -wl && p->w2 <= wl && p->w3 >= -wl && p->w3 <= wl, ICD2S_ERR_RANGE,
        "|w| must be <= 2^24 (Q16)");
    REQ(p->mut_mode == 0 || (p->mut_mode == 1 && p->mut_rate >= 0 && p->mut_rate <= 1), ICD2S_ERR_ARG,
        "mut_mode must be 0 or 1 with 0 <= mut_rate <= 1");
    REQ(p->max_iters >= 0, ICD2S_ERR_ARG, "max_iters < 0");
    REQ(p->select_mode >= 0 && p->select_mode <= 2, ICD2S_ERR_ARG, "select_mode=%d outside 0..2", p->select_mode);
    REQ(p->select_mode == 0 || st->mlp, ICD2S_ERR_STATE, "select_mode %d needs a network (icd2s_state_set_mlp)",
        p->select_mode);
    REQ(p->stop_at_target == 0 || p->stop_at_target == 1, ICD2S_ERR_ARG, "stop_at_target must be 0 or 1");
    REQ(p->im_mode == 0 || (p->im_mode == 1 && p->m_max <= 24 && mi <= 24), ICD2S_ERR_RANGE,
        "im_mode must be 0, or 1 (exact) with subQUBOs of at most 24 variables");
    REQ(p->ablation >= 0 && p->ablation <= 2, ICD2S_ERR_ARG, "ablation=%d outside 0..2", p->ablation);
    REQ(p->ablation == 0 || p->select_mode == 0, ICD2S_ERR_ARG, "the ablations use the paper's selection rule");
    REQ(p->aspiration == 0 || p->aspiration == 1, ICD2S_ERR_ARG, "aspiration must be 0 or 1");
    REQ(p->im_order == 0 || p->im_order == 1, ICD2S_ERR_ARG, "im_order must be 0 or 1");
    REQ(p->t_start >= 0 && p->t_start <= p->max_iters, ICD2S_ERR_ARG, "t_start=%d outside 0..max_iters=%d",
        p->t_start, p->max_iters);
    return ICD2S_OK;
}

extern "C" {

const char* icd2s_last_error(void) { return g_err; }

int32_t icd2s_version(void) { return 101; }

int icd2s_default_params(int32_t n, icd2s_params* out)
{
    REQ(out, ICD2S_ERR_ARG, "out is NULL");
    REQ(n >= 1 && n <= kMaxN, ICD2S_ERR_RANGE, "n=%d outside 1..%d", n, kMaxN);
    std::memset(out, 0, sizeof *out);
    const int m = n < 50 ? n : 50;
    int c = n / 150;
    if (c < 2) c = 2;
    if (c > n) c = n;
    out->z = 4; out->K = 1; out->m_min = m; out->m_max = m; out->m_init = m;
    out->alpha = 5 * n; out->c = c; out->sweeps = 256; out->T_max = 100.0; out->T_min = 1.0;
    out->w1 = 65536; out->w2 = 65536; out->w3 = 32768;
    out->mut_mode = 0; out->mut_rate = 0.0; out->patience = 30; out->max_iters = 100;
    return ICD2S_OK;
}

int icd2s_tables(int32_t sweeps, double T_max, double T_min, uint32_t* beta, uint32_t* nlog)
{
    REQ(sweeps >= 0, ICD2S_ERR_ARG, "sweeps < 0");
    if (beta && sweeps > 0) make_beta(sweeps, T_max, T_min, beta);
    if (nlog) make_nlog(nlog);
    return ICD2S_OK;
}

// ----------------------------------------------------------------------------- problem
int icd2s_qubo_create(const int8_t* Q_host, int32_t n, icd2s_qubo** out)
{
    REQ(Q_host && out, ICD2S_ERR_ARG, "NULL argument");
    *out = nullptr;
    REQ(n >= 1 && n <= kMaxN, ICD2S_ERR_RANGE, "n=%d outside 1..%d", n, kMaxN);
    auto* q = new icd2s_qubo();
    q->n = n;
    q->ld = round_up(n, kLdAlign);
    auto bail = [&](int code) {
        if (q->Q) cudaFree(q->Q);
        if (q->diag) cudaFree(q->diag);
        if (q->Q2) cudaFree(q->Q2);
        if (q->Qpk) cudaFree(q->Qpk);
        if (q->pk_perm) cudaFree(q->pk_perm);
        if (q->eta) cudaFree(q->eta);
        if (q->etahat) cudaFree(q->etahat);
        delete q;
        return code;
    };
    int* mism = nullptr;
    cudaError_t e;
    if ((e = dalloc(&q->Q, (size_t)n * q->ld)) != cudaSuccess || (e = dalloc(&q->diag, q->ld)) != cudaSuccess ||
        (e = dalloc(&q->eta, q->ld)) != cudaSuccess || (e = dalloc(&q->etahat, q->ld)) != cudaSuccess ||
        (e = dalloc(&mism, 4)) != cudaSuccess)
        return bail(fail(ICD2S_ERR_OOM, "device allocation failed: %s", cudaGetErrorString(e)));
    int got[4] = {0, 0, 0, 0};  // symmetry mismatches, max_j eta_j, entries equal to -128, max |g|
    if ((e = cudaMemset(q->Q, 0, (size_t)n * q->ld)) == cudaSuccess &&
        (e = cudaMemcpy2D(q->Q, q->ld, Q_host, n, n, n, cudaMemcpyHostToDevice)) == cudaSuccess &&
        (e = cudaMemset(mism, 0, 4 * sizeof(int))) == cudaSuccess &&
        (e = launch_prepare(q->Q, n, q->ld, q->eta, q->etahat, q->diag, mism, mism + 1, mism + 3, 0)) ==
            cudaSuccess &&
        (e = cudaMemcpy(got, mism, 4 * sizeof(int), cudaMemcpyDeviceToHost)) == cudaSuccess) {
        cudaFree(mism);
        mism = nullptr;
        const int bad = got[0];
        q->gain_bound = got[3];
        q->has_m128 = got[2] != 0;
        if (bad) return bail(fail(ICD2S_ERR_ASYMMETRIC, "Q is not symmetric (%d mismatched entries)", bad));
        // parity labels: the variables with an even diagonal, then the odd ones
        std::vector<int32_t> perm(n);
        int n0 = 0;
        for (int j = 0; j < n; ++j)
            if ((Q_host[(size_t)j * n + j] & 1) == 0) perm[n0++] = j;
        for (int j = 0, k = n0; j < n; ++j)
            if ((Q_host[(size_t)j * n + j] & 1) != 0) perm[k++] = j;
        if (tabu_key_shift(n, q->gain_bound) == 0 && tabu_key_shift_pk(n0, n - n0, q->gain_bound) > 0) {
            if ((e = dalloc(&q->Qpk, (size_t)n * q->ld)) != cudaSuccess || (e = dalloc(&q->pk_perm, n)) != cudaSuccess)
                return bail(fail(ICD2S_ERR_OOM, "device allocation failed: %s", cudaGetErrorString(e)));
            q->pk_n0 = n0;
            if ((e = cudaMemcpy(q->pk_perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = launch_relabel(q->Q, q->pk_perm, n, q->ld, q->Qpk, 0)) != cudaSuccess ||
                (e = cudaDeviceSynchronize()) != cudaSuccess)
                return bail(fail(ICD2S_ERR_CUDA, "qubo_create: %s", cudaGetErrorString(e)));
        }
        *out = q;
        return ICD2S_OK;
    }
    cudaFree(mism);
    return bail(fail(ICD2S_ERR_CUDA, "qubo_create: %s", cudaGetErrorString(e)));
}

int icd2s_qubo_destroy(icd2s_qubo* q)
{
    if (!q) return ICD2S_OK;
    void* ptrs[] = {q->Q, q->Q2, q->Qpk, q->pk_perm, q->diag, q->eta, q->etahat, q->xpad, q->hpad, q->Qb};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete q;
    return ICD2S_OK;
}

int icd2s_qubo_size(const icd2s_qubo* q, int32_t* n_out)
{
    REQ(q && n_out, ICD2S_ERR_ARG, "NULL argument");
    *n_out = q->n;
    return ICD2S_OK;
}

int icd2s_qubo_gain_bound(const icd2s_qubo* q, int64_t* bound_out)
{
    REQ(q && bound_out, ICD2S_ERR_ARG, "NULL argument");
    *bound_out = q->gain_bound;
    return ICD2S_OK;
}

int icd2s_energy(icd2s_qubo* q, const uint8_t* x_dev, int32_t count, int64_t* E_dev, void* stream)
{
    REQ(q && (count == 0 || (x_dev && E_dev)), ICD2S_ERR_ARG, "NULL argument");
    REQ(count >= 0, ICD2S_ERR_ARG, "count < 0");
    if (count == 0) return ICD2S_OK;
    cudaStream_t s = S(stream);
    if (count > q->cap) {
        CK(cudaStreamSynchronize(s));
        if (q->xpad) cudaFree(q->xpad);
        if (q->hpad) cudaFree(q->hpad);
        q->xpad = nullptr; q->hpad = nullptr; q->cap = 0;
        CK(dalloc(&q->xpad, (size_t)count * q->ld));
        CK(dalloc(&q->hpad, (size_t)count * q->ld));
        q->cap = count;
    }
    Dev d{};
    d.Q = q->Q; d.diag = q->diag; d.etahat = q->etahat; d.n = q->n; d.ld = q->ld; d.R = count;
    d.gain_bound = q->gain_bound;
    d.Q2 = nullptr;  // signed rows only once the state asks for them
    CK(launch_pad_rows(x_dev, q->n, count, q->xpad, q->ld, s));
    CK(launch_recompute(d, q->xpad, q->ld, count, q->hpad, E_dev, s));
    return ICD2S_OK;
}

// ----------------------------------------------------------------------------- solutions
int icd2s_state_create(icd2s_qubo* q, int32_t replicas, uint64_t seed, icd2s_state** out)
{
    return icd2s_state_create_shard(q, replicas, 0, replicas, seed, out);
}

int icd2s_state_create_shard(icd2s_qubo* q, int32_t replicas, int32_t replica_base, int32_t replicas_total,
                             uint64_t seed, icd2s_state** out)
{
    REQ(q && out, ICD2S_ERR_ARG, "NULL argument");
    *out = nullptr;
    REQ(replicas >= 1 && replicas <= kMaxReplicas, ICD2S_ERR_RANGE, "replicas=%d outside 1..%d", replicas,
        kMaxReplicas);
    REQ(replica_base >= 0 && (long long)replica_base + replicas <= replicas_total, ICD2S_ERR_ARG,
        "replicas %d..%d outside the set of %d", replica_base, replica_base + replicas - 1, replicas_total);
    auto* st = new icd2s_state();
    st->q = q; st->R = replicas; st->seed = seed;
    const size_t RL = (size_t)replicas * q->ld;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, cnt) if (e == cudaSuccess) e = dalloc(&st->ptr, (cnt))
    ALLOC(X, RL); ALLOC(G, RL); ALLOC(E, replicas); ALLOC(T, RL); ALLOC(C, RL); ALLOC(gamma, q->ld);
    ALLOC(A, RL); ALLOC(delta, RL); ALLOC(order, RL); ALLOC(sel, RL); ALLOC(FL, RL); ALLOC(FCNT, replicas);
    ALLOC(DEACC, replicas); ALLOC(DONE, replicas); ALLOC(best_x, q->ld); ALLOC(best_E, 1); ALLOC(flags, 8);
    ALLOC(idx, RL); ALLOC(off, (size_t)replicas * 64 + 1); ALLOC(scratch, RL); ALLOC(counters, 4);
    ALLOC(nlog, 4096); ALLOC(lpt, (size_t)replicas * 64); ALLOC(queue, 4); ALLOC(ctx, 4); ALLOC(H, RL);
    ALLOC(ACC, RL * apply_splits_for(q->ld, replicas)); ALLOC(TT, (size_t)replicas * apply_tiles(q->ld));
#undef ALLOC
    if (e != cudaSuccess) {
        free_state(st);
        return fail(ICD2S_ERR_OOM, "device allocation failed: %s", cudaGetErrorString(e));
    }
    Dev& d = st->d;
    d.Q = q->Q; d.diag = q->diag; d.etahat = q->etahat; d.n = q->n; d.ld = q->ld; d.R = replicas;
    d.gain_bound = q->gain_bound;
    d.Q2 = nullptr;  // signed rows only once the state asks for them
    d.Qpk = q->Qpk; d.pk_perm = q->pk_perm; d.pk_n0 = q->pk_n0;
    d.X = st->X; d.G = st->G; d.E = st->E; d.T = st->T; d.C = st->C; d.gamma = st->gamma; d.A = st->A;
    d.delta = st->delta; d.order = st->order; d.sel = st->sel; d.FL = st->FL; d.FCNT = st->FCNT;
    d.DEACC = st->DEACC; d.DONE = st->DONE; d.best_x = st->best_x; d.best_E = st->best_E; d.flags = st->flags;
    d.H = st->H;
    d.ACC = st->ACC; d.TT = st->TT; d.apply_splits = apply_splits_for(q->ld, replicas);
    d.k0 = (uint32_t)(seed & 0xffffffffu); d.k1 = (uint32_t)(seed >> 32);
    d.p0 = replica_base; d.z_total = replicas_total;
    uint32_t nl[4096];
    make_nlog(nl);
    const int64_t big = INT64_MAX;
    int rc = ICD2S_OK;
    if ((e = cudaMemset(st->T, 0, RL * 4)) != cudaSuccess || (e = cudaMemset(st->C, 0, RL * 4)) != cudaSuccess ||
        (e = cudaMemset(st->FCNT, 0, replicas * 4)) != cudaSuccess ||
        (e = cudaMemset(st->DEACC, 0, replicas * 8)) != cudaSuccess ||
        (e = cudaMemset(st->DONE, 0, replicas * 4)) != cudaSuccess || (e = cudaMemset(st->flags, 0, 32)) != cudaSuccess ||
        (e = cudaMemset(st->H, 0, RL * 4)) != cudaSuccess || 
        (e = cudaMemset(st->TT, 0, sizeof(unsigned) * replicas * apply_tiles(q->ld))) != cudaSuccess ||
        (e = cudaMemset(st->counters, 0, 32)) != cudaSuccess || (e = cudaMemset(st->best_x, 0, q->ld)) != cudaSuccess ||
        (e = cudaMemcpy(st->best_E, &big, 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(st->nlog, nl, sizeof nl, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = launch_init_x(d, 0)) != cudaSuccess || (e = launch_recompute(d, d.X, d.ld, d.R, d.G, d.E, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
        rc = fail(ICD2S_ERR_CUDA, "state_create: %s", cudaGetErrorString(e));
    if (rc != ICD2S_OK) { free_state(st); return rc; }
    *out = st;
    return ICD2S_OK;
}

int icd2s_state_destroy(icd2s_state* st)
{
    if (st) free_state(st);
    return ICD2S_OK;
}

int icd2s_state_load(icd2s_state* st, const uint8_t* x, int32_t x_is_device, void* stream)
{
    REQ(st && x, ICD2S_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    const int n = st->q->n, R = st->R;
    const uint8_t* src = x;
    if (!x_is_device) {
        CK(cudaMemcpyAsync(st->scratch, x, (size_t)R * n, cudaMemcpyHostToDevice, s));
        src = st->scratch;
    }
    CK(launch_pad_rows(src, n, R, st->X, st->q->ld, s));
    CK(launch_recompute(st->d, st->X, st->q->ld, R, st->G, st->E, s));
    CK(cudaMemsetAsync(st->H, 0, (size_t)R * st->q->ld * 4, s));
    return ICD2S_OK;
}

int icd2s_get_state(icd2s_state* st, uint8_t* x, int32_t* g, int64_t* E)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    CK(cudaDeviceSynchronize());
    if (x) CK(cudaMemcpy2D(x, n, st->X, ld, n, R, cudaMemcpyDeviceToHost));
    if (g) CK(cudaMemcpy2D(g, (size_t)n * 4, st->G, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    if (E) CK(cudaMemcpy(E, st->E, (size_t)R * 8, cudaMemcpyDeviceToHost));
    return ICD2S_OK;
}

int icd2s_get_best(icd2s_state* st, uint8_t* x_best, int64_t* E_best)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    CK(cudaDeviceSynchronize());
    if (x_best) CK(cudaMemcpy(x_best, st->best_x, st->q->n, cudaMemcpyDeviceToHost));
    if (E_best) CK(cudaMemcpy(E_best, st->best_E, 8, cudaMemcpyDeviceToHost));
    return ICD2S_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- checkpoint and resume
namespace {

constexpr char kCkMagic[8] = {'I', 'C', 'D', '2', 'S', 'C', 'K', 'P'};
constexpr uint32_t kCkVersion = 1;
constexpr size_t kCkHeader = 64;

// FNV-1a, 64-bit (Fowler, Noll, Vo): offset basis 14695981039346656037,
// prime 1099511628211; per byte, xor then multiply.
uint64_t fnv1a64(const unsigned char* p, size_t len)
{
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < len; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

template <class T>
T get_le(const unsigned char* p)
{
    T v;
    std::memcpy(&v, p, sizeof v);  // both supported hosts (x86-64, aarch64) are little-endian
    return v;
}

template <class T>
void put_le(unsigned char* p, T v) { std::memcpy(p, &v, sizeof v); }

uint64_t ck_payload(int n, int R) { return 5ull * (uint64_t)R * (uint64_t)n + (uint64_t)n; }

struct CkInfo { int32_t n, R, t_next, stale; uint64_t seed; int64_t best_E; };

// Every check of a checkpoint that needs no state; host only.
int ck_parse(const void* buf, size_t bytes, CkInfo* ci)
{
    REQ(buf, ICD2S_ERR_ARG, "checkpoint is NULL");
    const auto* b = static_cast<const unsigned char*>(buf);
    REQ(bytes >= kCkHeader + 8, ICD2S_ERR_ARG, "checkpoint of %zu bytes is shorter than its header", bytes);
    REQ(std::memcmp(b, kCkMagic, 8) == 0, ICD2S_ERR_ARG, "not a checkpoint (magic)");
    const uint32_t ver = get_le<uint32_t>(b + 8);
    REQ(ver == kCkVersion, ICD2S_ERR_ARG, "checkpoint version %u (this library reads %u)", ver, kCkVersion);
    CkInfo c{};
    c.n = get_le<int32_t>(b + 12); c.R = get_le<int32_t>(b + 16); c.t_next = get_le<int32_t>(b + 20);
    c.seed = get_le<uint64_t>(b + 24); c.best_E = get_le<int64_t>(b + 32); c.stale = get_le<int32_t>(b + 40);
    REQ(c.n >= 1 && c.n <= kMaxN && c.R >= 1 && c.R <= kMaxReplicas, ICD2S_ERR_ARG,
        "checkpoint sizes n=%d replicas=%d outside the library's limits", c.n, c.R);
    const uint64_t P = ck_payload(c.n, c.R);
    REQ(get_le<uint64_t>(b + 48) == P && bytes == kCkHeader + P + 8, ICD2S_ERR_ARG,
        "checkpoint of %zu bytes does not match n=%d, replicas=%d", bytes, c.n, c.R);
    REQ(get_le<uint32_t>(b + 44) == 0 && get_le<uint64_t>(b + 56) == 0, ICD2S_ERR_ARG,
        "checkpoint header fields that must be zero are not");
    REQ(fnv1a64(b, kCkHeader + P) == get_le<uint64_t>(b + kCkHeader + P), ICD2S_ERR_INVARIANT,
        "checkpoint checksum mismatch (corrupted)");
    REQ(c.t_next >= 0 && c.stale >= 0, ICD2S_ERR_ARG, "checkpoint t_next=%d stale=%d", c.t_next, c.stale);
    const unsigned char* x = b + kCkHeader;
    for (uint64_t k = 0; k < (uint64_t)c.R * c.n + c.n; ++k)
        REQ(x[k] <= 1, ICD2S_ERR_ARG, "checkpoint solution byte %llu is %u, not 0/1", (unsigned long long)k, x[k]);
    *ci = c;
    return ICD2S_OK;
}

}  // namespace

extern "C" {

int icd2s_state_save(icd2s_state* st, int32_t t_next, void* buf, size_t cap, size_t* bytes)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    REQ(t_next >= 0, ICD2S_ERR_ARG, "t_next=%d < 0", t_next);
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    const uint64_t P = ck_payload(n, R);
    const size_t total = kCkHeader + (size_t)P + 8;
    if (bytes) *bytes = total;
    if (!buf) return ICD2S_OK;
    REQ(cap >= total, ICD2S_ERR_RANGE, "checkpoint needs %zu bytes, buffer has %zu", total, cap);
    auto* b = static_cast<unsigned char*>(buf);
    int64_t bestE = 0;
    int32_t flags[2] = {0, 0};
    CK(cudaDeviceSynchronize());
    unsigned char* x = b + kCkHeader;
    unsigned char* bx = x + (size_t)R * n;
    unsigned char* h = bx + n;
    CK(cudaMemcpy2D(x, n, st->X, ld, n, R, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bx, st->best_x, n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy2D(h, (size_t)n * 4, st->H, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&bestE, st->best_E, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(flags, st->flags, 8, cudaMemcpyDeviceToHost));
    std::memcpy(b, kCkMagic, 8);
    put_le<uint32_t>(b + 8, kCkVersion);
    put_le<int32_t>(b + 12, n); put_le<int32_t>(b + 16, R); put_le<int32_t>(b + 20, t_next);
    put_le<uint64_t>(b + 24, st->seed); put_le<int64_t>(b + 32, bestE); put_le<int32_t>(b + 40, flags[1]);
    put_le<uint32_t>(b + 44, 0u); put_le<uint64_t>(b + 48, P); put_le<uint64_t>(b + 56, 0ull);
    put_le<uint64_t>(b + kCkHeader + P, fnv1a64(b, kCkHeader + (size_t)P));
    return ICD2S_OK;
}

int icd2s_checkpoint_info(const void* buf, size_t bytes, int32_t* n, int32_t* replicas, int32_t* t_next,
                          uint64_t* seed)
{
    CkInfo c{};
    const int rc = ck_parse(buf, bytes, &c);
    if (rc) return rc;
    if (n) *n = c.n;
    if (replicas) *replicas = c.R;
    if (t_next) *t_next = c.t_next;
    if (seed) *seed = c.seed;
    return ICD2S_OK;
}

int icd2s_state_restore(icd2s_state* st, const void* buf, size_t bytes, int32_t* t_next)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    CkInfo c{};
    const int rc = ck_parse(buf, bytes, &c);
    if (rc) return rc;
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    REQ(c.n == n && c.R == R, ICD2S_ERR_ARG, "checkpoint of n=%d, replicas=%d does not fit a state of n=%d, replicas=%d",
        c.n, c.R, n, R);
    const auto* x = static_cast<const unsigned char*>(buf) + kCkHeader;
    const unsigned char* bx = x + (size_t)R * n;
    const unsigned char* h = bx + n;
    cudaStream_t s = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(st->scratch, x, (size_t)R * n, cudaMemcpyHostToDevice));
    CK(launch_pad_rows(st->scratch, n, R, st->X, ld, s));
    CK(launch_recompute(st->d, st->X, ld, R, st->G, st->E, s));
    CK(cudaMemset(st->best_x, 0, ld));
    CK(cudaMemcpy(st->best_x, bx, n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(st->best_E, &c.best_E, 8, cudaMemcpyHostToDevice));
    // only the stale count carries over: no improvement-log entry is pending
    const int32_t fl[8] = {0, c.stale, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpy(st->flags, fl, sizeof fl, cudaMemcpyHostToDevice));
    CK(cudaMemset(st->H, 0, (size_t)R * ld * 4));
    CK(cudaMemcpy2D(st->H, (size_t)ld * 4, h, (size_t)n * 4, (size_t)n * 4, R, cudaMemcpyHostToDevice));
    st->seed = c.seed;
    st->d.k0 = (uint32_t)(c.seed & 0xffffffffu);
    st->d.k1 = (uint32_t)(c.seed >> 32);
    st->have_features = st->have_scores = false;
    ++st->gen;  // a captured step holds the old Philox key
    CK(cudaDeviceSynchronize());
    if (t_next) *t_next = c.t_next;
    return ICD2S_OK;
}

int icd2s_get_tabu(icd2s_state* st, int32_t* T, int32_t* C)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    CK(cudaDeviceSynchronize());
    if (T) CK(cudaMemcpy2D(T, (size_t)n * 4, st->T, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    if (C) CK(cudaMemcpy2D(C, (size_t)n * 4, st->C, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    return ICD2S_OK;
}

int icd2s_get_control(icd2s_state* st, int32_t* A, int32_t* gamma, int32_t* delta)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    REQ(st->have_select, ICD2S_ERR_STATE, "no selection has been made yet");
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    CK(cudaDeviceSynchronize());
    if (A) CK(cudaMemcpy2D(A, (size_t)n * 4, st->A, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    if (delta)
        CK(cudaMemcpy2D(delta, (size_t)n * 4, st->delta, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    if (gamma) CK(cudaMemcpy(gamma, st->gamma, (size_t)n * 4, cudaMemcpyDeviceToHost));
    return ICD2S_OK;
}

// Signed row pairs of the instance (2 n ld bytes beside Q), made the first time
// a state asks for them; none when Q has an entry -128.  The state's view is
// updated (a captured step holds the pointer, so gen moves on).
static int ensure_signed_rows(icd2s_state* st)
{
    icd2s_qubo* q = st->q;
    if (!q->Q2 && !q->has_m128) {
        CK(cudaDeviceSynchronize());
        int8_t* q2 = nullptr;
        cudaError_t e = dalloc(&q2, 2 * (size_t)q->n * q->ld);
        REQ(e == cudaSuccess, ICD2S_ERR_OOM, "signed rows: %s", cudaGetErrorString(e));
        if ((e = launch_signed_rows(q->Q, q->n, q->ld, q2, 0)) == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) cudaFree(q2);
        CK(e);
        q->Q2 = q2;  // only once it holds the rows
    }
    if (st->d.Q2 != q->Q2) {
        st->d.Q2 = q->Q2;
        ++st->gen;
    }
    return ICD2S_OK;
}

// ----------------------------------------------------------------------------- steps
// Move logs in global memory for Tabu searches whose log (2 bytes a move) does
// not fit shared memory beside the search's state: [R][alpha] uint16, made on
// first use and kept (a captured step holds the pointer, so a new buffer bumps gen).
static int ensure_tabu_log(icd2s_state* st, int alpha, cudaStream_t s)
{
    if (tabu_log_in_smem(st->q->n, alpha) || st->tlog_cap >= alpha) return ICD2S_OK;
    CK(cudaStreamSynchronize(s));
    if (st->tlog) {
        cudaFree(st->tlog);
        st->tlog = nullptr; st->tlog_cap = 0;
        st->d.TL = nullptr; st->d.tl_cap = 0;  // no launch may see the freed log
        ++st->gen;
    }
    cudaError_t e = dalloc(&st->tlog, (size_t)st->R * (size_t)alpha);
    REQ(e == cudaSuccess, ICD2S_ERR_OOM, "Tabu move log of %lld bytes: %s", 2LL * st->R * alpha, cudaGetErrorString(e));
    st->tlog_cap = alpha;
    st->d.TL = st->tlog;
    st->d.tl_cap = alpha;
    ++st->gen;
    return ICD2S_OK;
}

int icd2s_tabu(icd2s_state* st, int32_t alpha, int32_t c, void* stream)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    const int n = st->q->n;
    REQ(alpha >= 0, ICD2S_ERR_ARG, "alpha < 0");
    REQ(c >= 1 && c <= n, ICD2S_ERR_ARG, "tenure c=%d outside 1..n", c);
    int rc = ensure_tabu_log(st, alpha, S(stream));
    if (rc) return rc;
    CK(launch_tabu(st->d, alpha, c, st->tune.tabu_variant, S(stream), false, st->tune.tabu_wide_keys != 0,
                   st->tune.tabu_rows, st->tune.tabu_cluster));
    return ICD2S_OK;
}

int icd2s_tabu_aspiration(icd2s_state* st, int32_t alpha, int32_t c, void* stream)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    const int n = st->q->n;
    REQ(alpha >= 0, ICD2S_ERR_ARG, "alpha < 0");
    REQ(c >= 1 && c <= n, ICD2S_ERR_ARG, "tenure c=%d outside 1..n", c);
    int rc = ensure_tabu_log(st, alpha, S(stream));
    if (rc) return rc;
    CK(launch_tabu(st->d, alpha, c, st->tune.tabu_variant, S(stream), true, st->tune.tabu_wide_keys != 0,
                   st->tune.tabu_rows, st->tune.tabu_cluster));
    return ICD2S_OK;
}

// iter_dev: non-null when the iteration number comes from device memory (a replayed step).
// counts: the column counts of all replica shards for gamma (null: this
// state's own replicas, which must then be the whole set).
static int select_impl(icd2s_state* st, int64_t w1, int64_t w2, int64_t w3, int K, int m_min, int m_max,
                       uint32_t iter, cudaStream_t s, const int32_t* iter_dev = nullptr, int mode = 0,
                       bool count_hits = true, int ablation = 0, const int32_t* counts = nullptr)
{
    const int n = st->q->n;
    REQ(counts || st->d.z_total == st->R, ICD2S_ERR_STATE,
        "a replica shard takes gamma from the counts of every shard (icd2s_step_shard_finish)");
    REQ(K >= 1 && K <= 64, ICD2S_ERR_RANGE, "K=%d outside 1..64", K);
    REQ(m_min >= 1 && m_min <= m_max && m_max <= kMaxM, ICD2S_ERR_RANGE, "sizes %d..%d outside 1..256", m_min, m_max);
    if (ablation == 1) m_min = m_max = 0;  // No_IM: an empty subset (only A and its ranking are made)
    REQ((long long)K * m_max <= n, ICD2S_ERR_ARG, "K*m_max exceeds n");
    const int64_t wl = (int64_t)1 << 24;
    REQ(w1 >= -wl && w1 <= wl && w2 >= -wl && w2 <= wl && w3 >= -wl && w3 <= wl, ICD2S_ERR_RANGE, "|w| > 2^24");
    CK(launch_gamma(st->d, counts, s));
    CK(launch_sizes(st->R, K, m_min, m_max, st->d.k0, st->d.k1, iter, iter_dev, st->off, st->lpt, st->queue, s,
                    st->d.p0));
    CK(launch_select(st->d, w1, w2, w3, K, st->off, st->idx, mode, count_hits, s, iter, iter_dev, ablation));
    st->have_select = true;
    st->sel_K = K;
    return ICD2S_OK;
}

int icd2s_select_subqubos(icd2s_state* st, const icd2s_select_params* sp, int32_t* idx_dev, int32_t* off_dev,
                          void* stream)
{
    REQ(st && sp && idx_dev && off_dev, ICD2S_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    int rc = select_impl(st, sp->w1, sp->w2, sp->w3, sp->K, sp->m_min, sp->m_max, sp->iter, s);
    if (rc) return rc;
    const int cnt = st->R * sp->K;
    int total = 0;
    CK(cudaMemcpyAsync(&total, st->off + cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpyAsync(off_dev, st->off, sizeof(int) * (cnt + 1), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(idx_dev, st->idx, sizeof(int) * (size_t)total, cudaMemcpyDeviceToDevice, s));
    return ICD2S_OK;
}

// queued: the subQUBOs have uneven sizes and were ordered largest-first by
// the selection (st->lpt), so the persistent kernel takes them from its queue.
static int anneal_impl(icd2s_state* st, const int32_t* idx, const int32_t* off, int count, int per_replica,
                       int m_max, int block_m, int block_base, int sweeps, double T_max, double T_min, uint32_t iter,
                       uint8_t* mask, int ldm, int64_t* dE, cudaStream_t s, bool queued = false,
                       const int32_t* iter_dev = nullptr, int im_mode = 0, int group_k = -1)
{
    int rc = ensure_beta(st, sweeps, T_max, T_min, s);
    if (rc) return rc;
    AnnealArgs a{};
    a.idx = idx; a.off = off; a.count = count; a.per_replica = per_replica; a.block_m = block_m;
    a.block_base = block_base; a.limtab = st->limtab; a.sweeps = sweeps; a.iter = iter;
    // random streams by global replica: slot p K + k of a subQUBO, p of a block
    a.slot_base = (uint32_t)(idx ? st->d.p0 * per_replica : st->d.p0);
    a.mask = mask; a.ldm = ldm; a.dE = dE; a.attempts_acc = st->counters; a.m_max = m_max;
    a.warps_per_cta = st->tune.anneal_warps_per_cta;
    a.scheme = st->tune.anneal_scheme;
    a.iter_dev = iter_dev;
    if (group_k >= 0) { a.group_stride = per_replica; a.group_k = group_k; }  // count = replicas
    if (im_mode == 1) {  // exact Ising machine (m <= 24)
        CK(launch_exact(st->d, a, s));
        return ICD2S_OK;
    }
    if (queued) { a.queue = st->queue; a.order = st->lpt; }
    CK(launch_anneal(st->d, a, s));
    return ICD2S_OK;
}

int icd2s_exact_subqubos_batch(icd2s_state* st, const int32_t* idx_dev, const int32_t* off_dev, int32_t count,
                               int32_t per_replica, uint8_t* flips_dev, int64_t* dE_dev, void* stream)
{
    REQ(st && idx_dev && off_dev && flips_dev, ICD2S_ERR_ARG, "NULL argument");
    REQ(count >= 0, ICD2S_ERR_ARG, "count < 0");
    REQ(per_replica >= 1 && (long long)count <= (long long)st->R * per_replica, ICD2S_ERR_ARG,
        "count=%d exceeds replicas * per_replica", count);
    cudaStream_t s = S(stream);
    const int n = st->q->n;
    std::vector<int32_t> off((size_t)count + 1);
    CK(cudaMemcpyAsync(off.data(), off_dev, sizeof(int32_t) * (count + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int m_max = 1;
    for (int i = 0; i < count; ++i) {
        const int m = off[i + 1] - off[i];
        REQ(m >= 1 && m <= 24 && m <= n, ICD2S_ERR_RANGE, "subQUBO %d has size %d (exact: 1..24, <= n)", i, m);
        if (m > m_max) m_max = m;
    }
    CK(cudaMemsetAsync(flips_dev, 0, (size_t)st->R * n, s));
    return anneal_impl(st, idx_dev, off_dev, count, per_replica, m_max, 0, 0, 1, 1.0, 1.0, 0u, flips_dev, n, dE_dev,
                       s, false, nullptr, 1);
}

int icd2s_anneal_subqubos_batch(icd2s_state* st, const int32_t* idx_dev, const int32_t* off_dev, int32_t count,
                                const icd2s_anneal_params* ap, uint8_t* flips_dev, int64_t* dE_dev, void* stream)
{
    REQ(st && idx_dev && off_dev && ap && flips_dev, ICD2S_ERR_ARG, "NULL argument");
    REQ(count >= 0, ICD2S_ERR_ARG, "count < 0");
    REQ(ap->per_replica >= 1 && (long long)count <= (long long)st->R * ap->per_replica, ICD2S_ERR_ARG,
        "count=%d exceeds replicas * per_replica", count);
    REQ(ap->sweeps >= 1 && ap->T_min > 0 && ap->T_max >= ap->T_min, ICD2S_ERR_ARG, "bad anneal parameters");
    cudaStream_t s = S(stream);
    const int n = st->q->n;
    std::vector<int32_t> off((size_t)count + 1);
    CK(cudaMemcpyAsync(off.data(), off_dev, sizeof(int32_t) * (count + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int m_max = 1;
    for (int i = 0; i < count; ++i) {
        const int m = off[i + 1] - off[i];
        REQ(m >= 1 && m <= kMaxM && m <= n, ICD2S_ERR_RANGE, "subQUBO %d has size %d (allowed 1..256, <= n)", i, m);
        if (m > m_max) m_max = m;
    }
    CK(cudaMemsetAsync(flips_dev, 0, (size_t)st->R * n, s));
    return anneal_impl(st, idx_dev, off_dev, count, ap->per_replica, m_max, 0, 0, ap->sweeps, ap->T_max, ap->T_min,
                       ap->iter, flips_dev, n, dE_dev, s);
}

int icd2s_apply_flips_update_gains(icd2s_state* st, const uint8_t* flips_dev, void* stream)
{
    REQ(st && flips_dev, ICD2S_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    CK(launch_compact_mask(st->d, flips_dev, st->q->n, s));
    if (st->timing) {
        if (!st->aev[0]) for (cudaEvent_t& e : st->aev) CK(cudaEventCreate(&e));
        CK(cudaEventRecord(st->aev[0], s));
    }
    CK(launch_apply(st->d, s));
    if (st->timing) {
        CK(cudaEventRecord(st->aev[1], s));
        st->timed_apply = true;
    }
    return ICD2S_OK;
}

static int mutate_impl(icd2s_state* st, int mut_mode, double mut_rate, uint32_t iter, uint8_t* mask, cudaStream_t s)
{
    REQ(st->have_select, ICD2S_ERR_STATE, "mutate needs a selection (icd2s_select_subqubos) first");
    REQ(mut_mode == 0 || (mut_mode == 1 && mut_rate >= 0 && mut_rate <= 1), ICD2S_ERR_ARG, "bad mutation rate");
    const double r = mut_mode == 0 ? mutation_rate((int)iter) : mut_rate;
    if (mask) CK(cudaMemsetAsync(mask, 0, (size_t)st->R * st->q->n, s));
    CK(launch_mutate(st->d, st->sel_K, st->off, r, iter, nullptr, nullptr, mask, st->q->n, s));
    CK(launch_apply(st->d, s));
    return ICD2S_OK;
}

int icd2s_mutate(icd2s_state* st, const icd2s_mutate_params* mp, uint8_t* flips_dev, void* stream)
{
    REQ(st && mp, ICD2S_ERR_ARG, "NULL argument");
    return mutate_impl(st, mp->mut_mode, mp->mut_rate, mp->iter, flips_dev, S(stream));
}

int icd2s_refresh(icd2s_state* st, int32_t rebuild, int32_t* mismatches, void* stream)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    cudaStream_t s = S(stream);
    icd2s_qubo* q = st->q;
    const int n = q->n, ld = q->ld, R = st->R;
    const size_t RL = (size_t)R * ld;
    // operands: a BF16 copy of Q (default: measured faster), or Q as bytes converted
    // in shared memory (no copy: n * ld * 2 bytes less device memory)
    const bool bytes = st->tune.refresh_kind == 3;
    if (!bytes && !q->Qb) {
        CK(cudaStreamSynchronize(s));
        void* qb = nullptr;
        CK(dmalloc(&qb, (size_t)n * ld * 2));
        const cudaError_t e = launch_to_bf16(q->Q, true, (size_t)n * ld, qb, s);
        if (e != cudaSuccess) cudaFree(qb);
        CK(e);
        q->Qb = qb;  // only once it holds the converted matrix
    }
    if (!st->Xb) {
        CK(cudaStreamSynchronize(s));
        CK(dmalloc(&st->Xb, RL * 2));
    }
    if (!st->G2 || !st->E2 || !st->rflags) {  // all three or none
        CK(cudaStreamSynchronize(s));
        free_group(&st->G2, &st->E2, &st->rflags);
        cudaError_t e = dalloc(&st->G2, RL);
        if (e == cudaSuccess) e = dalloc(&st->E2, (size_t)R);
        if (e == cudaSuccess) e = dalloc(&st->rflags, 4);
        if (e != cudaSuccess) free_group(&st->G2, &st->E2, &st->rflags);
        CK(e);
    }
    CK(cudaMemsetAsync(st->rflags, 0, 16, s));
    CK(launch_to_bf16(st->X, false, RL, st->Xb, s));
    CK(cudaMemsetAsync(st->G2, 0, sizeof(int32_t) * RL, s));  // H accumulates split-K partial sums
    if (st->timing) {  // the events bracket the tensor-core kernel alone
        if (!st->rev[0]) for (cudaEvent_t& e : st->rev) CK(cudaEventCreate(&e));
        CK(cudaEventRecord(st->rev[0], s));
    }
    const int stall = st->refresh_stall > 0;
    const unsigned long long wait_ns = stall ? st->refresh_stall_wait_ns : 2000000000ull;
    if (stall) --st->refresh_stall;
    if (bytes)
        CK(launch_refresh_i8(q->Q, st->Xb, n, R, ld, st->G2, st->rflags, st->tune.refresh_bn,
                             st->tune.refresh_splits, wait_ns, stall, s));  // H into G2
    else
        CK(launch_refresh_mma(q->Qb, st->Xb, n, R, ld, st->G2, st->rflags, st->tune.refresh_bn,
                              st->tune.refresh_splits, st->tune.refresh_kind == 4 ? 256 : 128, wait_ns, stall, s));
    if (st->timing) {
        CK(cudaEventRecord(st->rev[1], s));
        st->timed_refresh = true;
    }
    CK(launch_finish_gains(q->diag, n, ld, st->X, st->G2, st->E2, R, s));     // H -> g, E
    CK(launch_compare(st->G, st->E, st->G2, st->E2, n, ld, R, st->rflags + 1, s));
    if (mismatches || rebuild) {
        // a timed-out pipeline leaves an incomplete sum: report it, and never
        // rebuild the state from it
        int f[2] = {0, 0};
        CK(cudaMemcpyAsync(f, st->rflags, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        REQ(f[0] == 0, ICD2S_ERR_TIMEOUT, "refresh: a tensor-core pipeline wait timed out");
        if (mismatches) *mismatches = f[1];
    }
    if (rebuild) {
        CK(cudaMemcpyAsync(st->G, st->G2, RL * 4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(st->E, st->E2, (size_t)R * 8, cudaMemcpyDeviceToDevice, s));
    }
    return ICD2S_OK;
}

int icd2s_best_update(icd2s_state* st, void* stream)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    CK(launch_best(st->d, nullptr, 0, nullptr, S(stream)));
    return ICD2S_OK;
}

int icd2s_initial_pass(icd2s_state* st, const icd2s_params* p, void* stream)
{
    REQ(st && p, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const int m = p->m_init > 0 ? p->m_init : p->m_max;
    if (p->ablation == 1) return ICD2S_OK;  // No_IM: no Ising-machine call at all
    // one block at a time (Gauss-Seidel); with K Ising machines per solution and the
    // Jacobi order, K consecutive blocks at once, each from the solution before the
    // group (reading S24)
    const int nb = st->q->n / m;
    const int G = (p->K > 1 && p->im_order == 0) ? p->K : 1;
    for (int l0 = 0; l0 < nb; l0 += G) {
        const int g = nb - l0 < G ? nb - l0 : G;
        rc = anneal_impl(st, nullptr, nullptr, st->R * g, g, m, m, l0 * m, p->sweeps, p->T_max, p->T_min,
                         0x80000000u | (uint32_t)l0, nullptr, 0, nullptr, s, false, nullptr, p->im_mode);
        if (rc) return rc;
        CK(launch_apply(st->d, s));
    }
    return ICD2S_OK;
}

// Feature, score and hit-count buffers of the learned selection (made on
// first use; a captured step holds the pointers, so a new buffer bumps gen).
static int ensure_features(icd2s_state* st, cudaStream_t s)
{
    if (st->F && st->score && st->gmax) return ICD2S_OK;
    const size_t RL = (size_t)st->R * st->q->ld;
    CK(cudaStreamSynchronize(s));
    free_group(&st->F, &st->score, &st->gmax);  // all three or none
    cudaError_t e = dalloc(&st->F, RL * 6);
    if (e == cudaSuccess) e = dalloc(&st->score, RL);
    if (e == cudaSuccess) e = dalloc(&st->gmax, (size_t)st->R);
    if (e != cudaSuccess) free_group(&st->F, &st->score, &st->gmax);
    CK(e);
    st->d.F = st->F;
    st->d.score = st->score;
    ++st->gen;
    return ICD2S_OK;
}

static bool wants_features(const icd2s_state* st, const icd2s_params* p)
{
    return p->select_mode != 0 || st->log_cap > 0;
}

// One outer iteration.  dev_iter: the kernels read t (and the mutation rate)
// from st->ctx / st->rates, and the last one advances st->ctx[0] -- the form
// that is captured once and replayed as a CUDA graph.  It runs in two parts:
// the Tabu search (and the learned selection's features and scores), then
// everything from the selection on, which needs gamma over all replicas; a
// replica shard runs them as icd2s_step_shard_begin / _finish with the
// column counts of every shard added up in between.
static int step_first(icd2s_state* st, const icd2s_params* p, int t, int64_t* trace_it, cudaStream_t s,
                      bool dev_iter = false)
{
    const int R = st->R;
    const int32_t* it_dev = dev_iter ? st->ctx : nullptr;
    int rc = ensure_beta(st, p->sweeps, p->T_max, p->T_min, s);
    if (rc) return rc;
    if ((rc = ensure_tabu_log(st, p->alpha, s))) return rc;  // (made before any capture by graph_step)
    const bool feats = wants_features(st, p);
    if (feats && (rc = ensure_features(st, s))) return rc;
    mark(st, 0, 0, s);
    CK(launch_tabu(st->d, p->alpha, p->c, st->tune.tabu_variant, s, p->aspiration != 0,
                   st->tune.tabu_wide_keys != 0, st->tune.tabu_rows, st->tune.tabu_cluster));  // Algorithm 1
    mark(st, 0, 1, s);
    CK(launch_best(st->d, trace_it, 0, dev_iter ? st->ctx : nullptr, s, nullptr, 0, t));
    mark(st, 1, 0, s);
    if (feats) {                                                   // learned selection: features, scores
        CK(launch_features(st->d, t, it_dev, p->alpha, p->c, st->gmax, s));
        st->have_features = true;
        if (st->mlp) {
            CK(launch_score(st->F, (long long)R * st->q->ld, st->mlp->Wb, st->score, s));
            st->have_scores = true;
        }
    }
    return ICD2S_OK;
}

// counts: gamma's column counts over every replica shard (null: this state's replicas)
static int step_second(icd2s_state* st, const icd2s_params* p, int t, int64_t* trace_it, cudaStream_t s,
                       bool dev_iter = false, const int32_t* counts = nullptr)
{
    const int R = st->R;
    const int32_t* it_dev = dev_iter ? st->ctx : nullptr;
    const bool queued = p->K > 1 || p->m_min != p->m_max;  // uneven batch: persistent queue kernel
    int rc = select_impl(st, p->w1, p->w2, p->w3, p->K, p->m_min, p->m_max, (uint32_t)t, s, it_dev,
                         p->select_mode, true, p->ablation, counts);                        // Eq. 6-8, Alg. 3-4
    if (rc) return rc;
    mark(st, 1, 1, s);
    mark(st, 2, 0, s);
    if (p->ablation != 1 && p->im_order == 1 && p->K > 1) {
        // Gauss-Seidel: group k of every replica, written back before group k + 1 is built
        for (int k = 0; k < p->K; ++k) {
            rc = anneal_impl(st, st->idx, st->off, R, p->K, p->m_max, 0, 0, p->sweeps, p->T_max, p->T_min,
                             (uint32_t)t, nullptr, 0, nullptr, s, false, it_dev, p->im_mode, k);
            if (rc) return rc;
            if (k + 1 < p->K) CK(launch_apply(st->d, s));
        }
    } else if (p->ablation != 1) {                                                          // No_IM skips the IM
        rc = anneal_impl(st, st->idx, st->off, R * p->K, p->K, p->m_max, 0, 0, p->sweeps, p->T_max, p->T_min,
                         (uint32_t)t, nullptr, 0, nullptr, s, queued, it_dev, p->im_mode);  // Eq. 4, Algorithm 4
        if (rc) return rc;
    }
    mark(st, 2, 1, s);
    mark(st, 3, 0, s);
    CK(launch_apply(st->d, s));
    mark(st, 3, 1, s);
    CK(launch_best(st->d, trace_it ? trace_it + R : nullptr, 0, dev_iter ? st->ctx : nullptr, s, nullptr, 1, t));
    const double r = p->mut_mode == 0 ? mutation_rate(t) : p->mut_rate;        // Eq. 5
    mark(st, 4, 0, s);
    CK(launch_mutate(st->d, st->sel_K, st->off, r, (uint32_t)t, it_dev, st->rates, nullptr, st->q->n, s,
                     p->ablation == 2));
    mark(st, 4, 1, s);
    mark(st, 5, 0, s);
    CK(launch_apply(st->d, s));
    mark(st, 5, 1, s);
    mark(st, 6, 0, s);
    CK(launch_best(st->d, trace_it ? trace_it + 2 * R : nullptr, 1, dev_iter ? st->ctx : nullptr, s,
                   st->log_cap > 0 ? st->log_ctl : nullptr, 2, t));
    if (st->log_cap > 0) CK(launch_log(st->d, st->prev_x, st->LF, st->LY, st->lrep, s));
    mark(st, 6, 1, s);
    st->timed_step = st->timing;
    return ICD2S_OK;
}

static int step_impl(icd2s_state* st, const icd2s_params* p, int t, int64_t* trace_it, cudaStream_t s,
                     bool dev_iter = false)
{
    int rc = step_first(st, p, t, trace_it, s, dev_iter);
    if (rc) return rc;
    return step_second(st, p, t, trace_it, s, dev_iter);
}

// Replays the outer iteration as one CUDA graph, capturing it first when
// there is no graph yet or the parameters, tuning or buffers changed.
static int graph_step(icd2s_state* st, const icd2s_params* p, int t, cudaStream_t caller)
{
    int rc = ensure_beta(st, p->sweeps, p->T_max, p->T_min, caller);
    if (rc) return rc;
    rc = ensure_rates(st, p->mut_mode, p->mut_rate, t + 1, caller);
    if (rc) return rc;
    if ((rc = ensure_tabu_log(st, p->alpha, caller))) return rc;
    cudaStream_t s = caller;
    if (!s) {  // the legacy stream cannot be captured: run on a private stream joined to it
        if (!st->own_stream) CK(cudaStreamCreateWithFlags(&st->own_stream, cudaStreamNonBlocking));
        if (!st->join_ev) CK(cudaEventCreateWithFlags(&st->join_ev, cudaEventDisableTiming));
        s = st->own_stream;
        CK(cudaEventRecord(st->join_ev, caller));
        CK(cudaStreamWaitEvent(s, st->join_ev, 0));
    }
    if (wants_features(st, p) && (rc = ensure_features(st, caller))) return rc;
    if (!st->graph || st->graph_gen != st->gen || std::memcmp(&st->graph_p, p, sizeof *p) != 0) {
        if (st->graph) { cudaGraphExecDestroy(st->graph); st->graph = nullptr; }
        const bool timing = st->timing;
        st->timing = false;  // no event records inside the graph
        const unsigned long long before = g_launches.load();
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        rc = step_impl(st, p, 0, nullptr, s, true);
        st->timing = timing;
        st->graph_kernels = g_launches.load() - before;  // captured, not run: counted per replay
        g_launches.fetch_sub(st->graph_kernels);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        CK(ec);
        const cudaError_t ei = cudaGraphInstantiate(&st->graph, g, 0);
        cudaGraphDestroy(g);
        CK(ei);
        st->graph_p = *p;
        st->graph_gen = st->gen;
        st->dev_t = -1;
    }
    if (st->dev_t != t) CK(launch_set_iter(st->ctx, t, s));
    CK(cudaGraphLaunch(st->graph, s));
    note_launch((int)st->graph_kernels);
    st->dev_t = t + 1;
    st->timed_step = false;
    if (!caller) {
        CK(cudaEventRecord(st->join_ev, s));
        CK(cudaStreamWaitEvent(caller, st->join_ev, 0));
    }
    return ICD2S_OK;
}

int icd2s_set_timing(icd2s_state* st, int32_t enable)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    if (enable && !st->ev[0])
        for (cudaEvent_t& e : st->ev) CK(cudaEventCreate(&e));
    st->timing = enable != 0;
    st->timed_step = false;
    return ICD2S_OK;
}

int icd2s_get_phase_ms(icd2s_state* st, double* ms)
{
    REQ(st && ms, ICD2S_ERR_ARG, "NULL argument");
    REQ(st->timed_step, ICD2S_ERR_STATE, "no timed step: enable icd2s_set_timing, then run icd2s_step");
    CK(cudaEventSynchronize(st->ev[2 * ICD2S_PHASES - 1]));
    for (int ph = 0; ph < ICD2S_PHASES; ++ph) {
        float f = 0.f;
        CK(cudaEventElapsedTime(&f, st->ev[2 * ph], st->ev[2 * ph + 1]));
        ms[ph] = f;
    }
    return ICD2S_OK;
}

int icd2s_get_refresh_ms(icd2s_state* st, double* ms)
{
    REQ(st && ms, ICD2S_ERR_ARG, "NULL argument");
    REQ(st->timed_refresh, ICD2S_ERR_STATE, "no timed refresh: enable icd2s_set_timing, then run icd2s_refresh");
    CK(cudaEventSynchronize(st->rev[1]));
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, st->rev[0], st->rev[1]));
    *ms = f;
    return ICD2S_OK;
}

int icd2s_get_apply_ms(icd2s_state* st, double* ms)
{
    REQ(st && ms, ICD2S_ERR_ARG, "NULL argument");
    REQ(st->timed_apply, ICD2S_ERR_STATE,
        "no timed write-back: enable icd2s_set_timing, then call icd2s_apply_flips_update_gains");
    CK(cudaEventSynchronize(st->aev[1]));
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, st->aev[0], st->aev[1]));
    *ms = f;
    return ICD2S_OK;
}

int icd2s_set_tuning(icd2s_state* st, const icd2s_tuning* t)
{
    REQ(st && t, ICD2S_ERR_ARG, "NULL argument");
    REQ(t->tabu_cluster == 0 || t->tabu_cluster == 1 || t->tabu_cluster == 2 || t->tabu_cluster == 4, ICD2S_ERR_ARG,
        "tabu_cluster=%d must be 0, 1, 2 or 4", t->tabu_cluster);
    REQ(t->tabu_variant < 0 || tabu_variant_fits(t->tabu_variant, st->q->n, t->tabu_cluster > 1 ? t->tabu_cluster : 1),
        ICD2S_ERR_ARG, "Tabu variant %d does not cover n=%d with %d CTAs per replica", t->tabu_variant, st->q->n,
        t->tabu_cluster > 1 ? t->tabu_cluster : 1);
    REQ(t->refresh_bn == 0 || t->refresh_bn == 128 || t->refresh_bn == 256, ICD2S_ERR_ARG,
        "refresh_bn=%d must be 0, 128 or 256", t->refresh_bn);
    REQ(t->refresh_splits >= 0 && t->refresh_splits <= 256, ICD2S_ERR_ARG, "refresh_splits=%d outside 0..256",
        t->refresh_splits);
    REQ(t->refresh_kind == 0 || t->refresh_kind == 1 || t->refresh_kind == 3 || t->refresh_kind == 4, ICD2S_ERR_ARG,
        "refresh_kind=%d must be 0, 1, 3 or 4", t->refresh_kind);
    REQ(t->anneal_warps_per_cta >= 0 && t->anneal_warps_per_cta <= 4, ICD2S_ERR_ARG,
        "anneal_warps_per_cta=%d outside 0..4", t->anneal_warps_per_cta);
    REQ(t->tabu_wide_keys == 0 || t->tabu_wide_keys == 1, ICD2S_ERR_ARG, "tabu_wide_keys=%d must be 0 or 1",
        t->tabu_wide_keys);
    REQ(t->tabu_rows >= 0 && t->tabu_rows <= 2, ICD2S_ERR_ARG, "tabu_rows=%d must be 0, 1 or 2", t->tabu_rows);
    if (t->tabu_rows == 2) {
        const int rc = ensure_signed_rows(st);
        if (rc) return rc;
    }
    REQ(t->anneal_scheme >= 0 && t->anneal_scheme <= 4, ICD2S_ERR_ARG, "anneal_scheme=%d outside 0..4",
        t->anneal_scheme);
    st->tune = *t;
    ++st->gen;  // launch configurations changed: re-capture
    return ICD2S_OK;
}

int icd2s_get_tuning(icd2s_state* st, icd2s_tuning* t)
{
    REQ(st && t, ICD2S_ERR_ARG, "NULL argument");
    *t = st->tune;
    return ICD2S_OK;
}

// Times the variants on the live workload.  The solutions are backed up in
// temporary buffers and restored after every trial; the trial selection
// overwrites the last one, so the caller must select again before
// icd2s_mutate.
int icd2s_autotune(icd2s_state* st, const icd2s_params* p, icd2s_tuning* chosen, void* stream)
{
    REQ(st && p, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    rc = ensure_beta(st, p->sweeps, p->T_max, p->T_min, s);
    if (rc) return rc;
    const int R = st->R, ld = st->q->ld, n = st->q->n;
    const size_t RL = (size_t)R * ld;
    uint8_t* xb = nullptr;
    int32_t* gb = nullptr;
    int64_t* eb = nullptr;
    struct Backup { uint8_t*& x; int32_t*& g; int64_t*& e;
        ~Backup() { if (x) cudaFree(x); if (g) cudaFree(g); if (e) cudaFree(e); } } backup{xb, gb, eb};
    CK(cudaStreamSynchronize(s));
    CK(dalloc(&xb, RL));
    CK(dalloc(&gb, RL));
    CK(dalloc(&eb, (size_t)R));
    CK(cudaMemcpyAsync(xb, st->X, RL, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(gb, st->G, RL * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(eb, st->E, (size_t)R * 8, cudaMemcpyDeviceToDevice, s));
    auto restore = [&]() -> int {
        CK(cudaMemcpyAsync(st->X, xb, RL, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(st->G, gb, RL * 4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(st->E, eb, (size_t)R * 8, cudaMemcpyDeviceToDevice, s));
        return ICD2S_OK;
    };
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
    icd2s_tuning best = st->tune;
    const int alpha = p->alpha < 2000 ? p->alpha : 2000;
    float best_ms = 1e30f;
    // CTAs per replica: one, and the splits that keep every CTA on an SM of its own
    // (a split needs the compact keys)
    const bool ck = st->tune.tabu_wide_keys == 0 && tabu_key_shift(n, st->d.gain_bound) > 0;
    for (int G : {1, 2, 4}) {
        if (G > 1 && (!ck || (long long)R * G > device_sm_count())) continue;
        for (int v = 0; v < tabu_num_variants(); ++v) {
            if (!tabu_variant_fits(v, n, G)) continue;
            for (int rows = 1; rows <= (st->d.Q2 ? 2 : 1); ++rows) {  // plain rows, then signed rows (if made)
                float vbest = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    if ((rc = restore())) return rc;
                    CK(cudaEventRecord(e0, s));
                    CK(launch_tabu(st->d, alpha, p->c, v, s, p->aspiration != 0, st->tune.tabu_wide_keys != 0, rows,
                                   G));
                    CK(cudaEventRecord(e1, s));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < vbest) vbest = ms;
                }
                if (vbest < best_ms) {
                    best_ms = vbest;
                    best.tabu_variant = v;
                    best.tabu_rows = rows;
                    best.tabu_cluster = G;
                }
            }
        }
    }
    if ((rc = restore())) return rc;
    rc = select_impl(st, p->w1, p->w2, p->w3, p->K, p->m_min, p->m_max, 0u, s, nullptr, 0, false);
    if (rc) return rc;
    AnnealArgs a{};
    a.idx = st->idx; a.off = st->off; a.count = R * p->K; a.per_replica = p->K; a.limtab = st->limtab;
    a.sweeps = p->sweeps < 128 ? p->sweeps : 128; a.iter = 0; a.mask = st->scratch; a.ldm = ld; a.m_max = p->m_max;
    best_ms = 1e30f;
    const int max_wpb = p->m_max > 128 ? 3 : 4;
    for (int w = 1; w <= max_wpb; ++w) {
        a.warps_per_cta = w;
        float vbest = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, s));
            CK(launch_anneal(st->d, a, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < vbest) vbest = ms;
        }
        if (vbest < best_ms) { best_ms = vbest; best.anneal_warps_per_cta = w; }
    }
    if ((rc = restore())) return rc;
    CK(cudaStreamSynchronize(s));
    st->have_select = false;
    st->tune = best;
    ++st->gen;
    if (chosen) *chosen = best;
    return ICD2S_OK;
}

int icd2s_kernel_launches(uint64_t* count)
{
    REQ(count, ICD2S_ERR_ARG, "NULL argument");
    *count = g_launches.load();
    return ICD2S_OK;
}

int icd2s_debug_refresh_stall(icd2s_state* st, int32_t launches, int32_t wait_us)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    REQ(launches >= 0 && wait_us >= 1 && wait_us <= 2000000, ICD2S_ERR_ARG,
        "launches=%d must be >= 0 and wait_us=%d in 1..2000000", launches, wait_us);
    st->refresh_stall = launches;
    st->refresh_stall_wait_ns = (unsigned long long)wait_us * 1000ull;
    return ICD2S_OK;
}

int icd2s_debug_fail_allocations_after(int32_t count)
{
    g_alloc_left.store(count < 0 ? -1 : (long long)count);
    return ICD2S_OK;
}

int icd2s_step(icd2s_state* st, const icd2s_params* p, int32_t t, void* stream)
{
    REQ(st && p, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    REQ(t >= 0, ICD2S_ERR_ARG, "t < 0");
    return p->use_graph ? graph_step(st, p, t, S(stream)) : step_impl(st, p, t, nullptr, S(stream));
}

int icd2s_im_round(icd2s_state* st, const icd2s_params* p, int32_t t, void* stream)
{
    REQ(st && p, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    REQ(t >= 0, ICD2S_ERR_ARG, "t < 0");
    REQ(p->ablation == 0, ICD2S_ERR_ARG, "an Ising-machine round has no ablation");
    cudaStream_t s = S(stream);
    if ((rc = ensure_beta(st, p->sweeps, p->T_max, p->T_min, s))) return rc;
    const bool feats = wants_features(st, p);
    if (feats) {
        REQ(st->have_scores, ICD2S_ERR_STATE, "the learned selection needs a step that scored the variables");
    }
    rc = select_impl(st, p->w1, p->w2, p->w3, p->K, p->m_min, p->m_max, (uint32_t)t, s, nullptr, p->select_mode,
                     true, 0);                                                              // Eq. 6-8, Alg. 3-4
    if (rc) return rc;
    const bool queued = p->K > 1 || p->m_min != p->m_max;
    rc = anneal_impl(st, st->idx, st->off, st->R * p->K, p->K, p->m_max, 0, 0, p->sweeps, p->T_max, p->T_min,
                     (uint32_t)t, nullptr, 0, nullptr, s, queued, nullptr, p->im_mode);  // Eq. 4, Algorithm 4
    if (rc) return rc;
    CK(launch_apply(st->d, s));
    return ICD2S_OK;
}

int icd2s_step_shard_begin(icd2s_state* st, const icd2s_params* p, int32_t t, int32_t* counts_dev, void* stream)
{
    REQ(st && p && counts_dev, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    REQ(t >= 0, ICD2S_ERR_ARG, "t < 0");
    cudaStream_t s = S(stream);
    if ((rc = step_first(st, p, t, nullptr, s))) return rc;
    CK(launch_colsum(st->d, counts_dev, s));
    return ICD2S_OK;
}

int icd2s_step_shard_finish(icd2s_state* st, const icd2s_params* p, int32_t t, const int32_t* counts_dev,
                            void* stream)
{
    REQ(st && p && counts_dev, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    REQ(t >= 0, ICD2S_ERR_ARG, "t < 0");
    return step_second(st, p, t, nullptr, S(stream), false, counts_dev);
}

int icd2s_get_best_info(icd2s_state* st, int64_t* E_best, int32_t* replica, int32_t* stamp)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    int64_t e = 0;
    int32_t f[8] = {};
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&e, st->best_E, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(f, st->flags, sizeof f, cudaMemcpyDeviceToHost));
    const bool any = e != INT64_MAX;
    if (E_best) *E_best = e;
    if (replica) *replica = any ? st->d.p0 + f[3] : -1;
    if (stamp) *stamp = any ? f[7] : -1;
    return ICD2S_OK;
}

int icd2s_step_host(icd2s_state* st, const icd2s_params* p, int32_t t, const uint8_t* x_in, uint8_t* x_out,
                    int64_t* E_out, void* stream)
{
    REQ(st && p, ICD2S_ERR_ARG, "NULL argument");
    int rc = check_params(st, p);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    if (x_in) {
        CK(cudaMemcpyAsync(st->scratch, x_in, (size_t)R * n, cudaMemcpyHostToDevice, s));
        CK(launch_pad_rows(st->scratch, n, R, st->X, ld, s));
        CK(launch_recompute(st->d, st->X, ld, R, st->G, st->E, s));
    }
    rc = p->use_graph ? graph_step(st, p, t, s) : step_impl(st, p, t, nullptr, s);
    if (rc) return rc;
    if (x_out) CK(cudaMemcpy2DAsync(x_out, n, st->X, ld, n, R, cudaMemcpyDeviceToHost, s));
    if (E_out) CK(cudaMemcpyAsync(E_out, st->E, (size_t)R * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ICD2S_OK;
}

// Algorithm 2 on a state: Call_IM_Solution_Set, then outer iterations until
// max_iters, patience or the target.  Per-iteration host synchronisation only
// when patience or the target needs this iteration's flags / best energy.
// t_start > 0 resumes a restored state at that iteration: no initial pass,
// its best solution and stale count carry on.
static int run_impl(icd2s_state* st, const icd2s_params* p, uint8_t* x_out, int64_t* E_out, icd2s_stats* stats,
                    int64_t* trace, uint8_t* S_out)
{
    int rc = check_params(st, p);
    if (rc) return rc;
    icd2s_qubo* q = st->q;
    const int R = st->R;
    struct Guard { int64_t* tr = nullptr; cudaEvent_t e0 = nullptr, e1 = nullptr, eh = nullptr; ~Guard() {
        if (tr) cudaFree(tr);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (eh) cudaEventDestroy(eh); } } guard;
    const size_t tr_len = (size_t)(p->max_iters > 0 ? p->max_iters : 1) * (3 * R + 1);
    if (trace) CK(dalloc(&guard.tr, tr_len));
    CK(cudaEventCreate(&guard.e0));
    CK(cudaEventCreate(&guard.e1));
    CK(cudaEventCreate(&guard.eh));
    cudaStream_t s = 0;
    const int t0 = p->t_start;
    if (t0 == 0) {
        const int64_t big = INT64_MAX;
        CK(cudaMemcpyAsync(st->best_E, &big, 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(st->flags, 0, 32, s));
        CK(cudaStreamSynchronize(s));  // the host value must stay alive
    }
    CK(cudaEventRecord(guard.e0, s));
    if (t0 == 0) {
        rc = icd2s_initial_pass(st, p, s);
        if (rc) return rc;
        CK(launch_best(st->d, nullptr, 0, nullptr, s));
        CK(cudaMemsetAsync(st->flags, 0, 8, s));
    }
    if (st->log_cap > 0) CK(cudaMemcpyAsync(st->prev_x, st->best_x, q->ld, cudaMemcpyDeviceToDevice, s));
    int64_t init_best = 0;
    int32_t flags[2] = {0, 0};  // [1]: iterations without a new best (a resumed run's carries on)
    CK(cudaMemcpyAsync(&init_best, st->best_E, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(flags, st->flags, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));  // init_best and flags are read below
    int t = t0, hit_iter = -1;
    if (p->stop_at_target && init_best <= p->target_E) {
        hit_iter = t0;
        CK(cudaEventRecord(guard.eh, s));
    }
    int64_t cur_best = init_best;
    const bool graph = p->use_graph && !trace;
    const bool sync_each = p->patience > 0 || p->stop_at_target;
    while (hit_iter < 0 && t < p->max_iters && (p->patience <= 0 || flags[1] < p->patience)) {
        if (graph) rc = graph_step(st, p, t, s);
        else rc = step_impl(st, p, t, guard.tr ? guard.tr + (size_t)t * (3 * R + 1) : nullptr, s);
        if (rc) return rc;
        if (p->refresh_every > 0 && (t + 1) % p->refresh_every == 0) {  // drift check on the tensor cores
            int32_t bad = 0;
            rc = icd2s_refresh(st, 0, &bad, s);
            if (rc) return rc;
            REQ(bad == 0, ICD2S_ERR_INVARIANT, "tracked gains/energies differ from the refresh in %d entries", bad);
        }
        ++t;
        if (sync_each) {  // the termination tests need this iteration's stale count / best energy
            CK(cudaEventRecord(guard.eh, s));
            CK(cudaMemcpyAsync(flags, st->flags, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&cur_best, st->best_E, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (p->stop_at_target && cur_best <= p->target_E) hit_iter = t;
        }
    }
    CK(cudaEventRecord(guard.e1, s));
    CK(cudaStreamSynchronize(s));
    int64_t bestE = 0;
    CK(cudaMemcpy(&bestE, st->best_E, 8, cudaMemcpyDeviceToHost));
    if (x_out) CK(cudaMemcpy(x_out, st->best_x, q->n, cudaMemcpyDeviceToHost));
    if (E_out) *E_out = bestE;
    if (trace && t > t0) {  // rows t0 .. t - 1 (a resumed run leaves the earlier rows untouched)
        const size_t row = (size_t)(3 * R + 1);
        CK(cudaMemcpy(trace + (size_t)t0 * row, guard.tr + (size_t)t0 * row, sizeof(int64_t) * (size_t)(t - t0) * row,
                      cudaMemcpyDeviceToHost));
    }
    if (S_out) CK(cudaMemcpy2D(S_out, q->n, st->X, q->ld, q->n, R, cudaMemcpyDeviceToHost));
    if (stats) {
        int64_t att = 0;
        CK(cudaMemcpy(&att, st->counters, 8, cudaMemcpyDeviceToHost));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, guard.e0, guard.e1));
        stats->iters = t; stats->best_E = bestE; stats->init_best_E = init_best; stats->anneal_attempts = att;
        stats->tabu_moves = (int64_t)(t - t0) * R * p->alpha; stats->device_ms = ms;
        stats->hit_iter = hit_iter;
        stats->ttt_ms = -1.0;
        if (hit_iter >= 0) {
            float mh = 0;
            CK(cudaEventElapsedTime(&mh, guard.e0, guard.eh));
            stats->ttt_ms = mh;
        }
    }
    return ICD2S_OK;
}

int icd2s_run(icd2s_qubo* q, const icd2s_params* p, uint64_t seed, uint8_t* x_out, int64_t* E_out,
              icd2s_stats* stats, int64_t* trace, uint8_t* S_out)
{
    REQ(q && p, ICD2S_ERR_ARG, "NULL argument");
    REQ(p->z >= 1 && p->z <= kMaxReplicas, ICD2S_ERR_RANGE, "z=%d outside 1..%d", p->z, kMaxReplicas);
    REQ(p->select_mode == 0, ICD2S_ERR_STATE, "learned selection needs a state with a network: icd2s_state_run");
    REQ(p->t_start == 0, ICD2S_ERR_ARG, "t_start > 0 resumes a restored state: icd2s_state_run");
    icd2s_state* st = nullptr;
    int rc = icd2s_state_create(q, p->z, seed, &st);
    if (rc) return rc;
    rc = run_impl(st, p, x_out, E_out, stats, trace, S_out);
    icd2s_state_destroy(st);
    return rc;
}

int icd2s_state_run(icd2s_state* st, const icd2s_params* p, uint8_t* x_out, int64_t* E_out, icd2s_stats* stats,
                    int64_t* trace, uint8_t* S_out)
{
    REQ(st && p, ICD2S_ERR_ARG, "NULL argument");
    return run_impl(st, p, x_out, E_out, stats, trace, S_out);
}

// ----------------------------------------------------------------------------- learned selection
static int mlp_upload(icd2s_mlp* m, const float* W)
{
    CK(cudaMemcpy(m->master, W, sizeof(float) * kNPar, cudaMemcpyHostToDevice));
    CK(cudaMemset(m->mom, 0, sizeof(float) * kNPar));
    CK(cudaMemset(m->vel, 0, sizeof(float) * kNPar));
    CK(launch_round_bf16(m->master, m->Wb, 0));
    CK(cudaDeviceSynchronize());
    m->adam_t = 0;
    return ICD2S_OK;
}

static void free_mlp(icd2s_mlp* m)
{
    void* ptrs[] = {m->master, m->mom, m->vel, m->Wb, m->partial, m->losses};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

int icd2s_mlp_create(uint64_t seed, icd2s_mlp** out)
{
    REQ(out, ICD2S_ERR_ARG, "NULL argument");
    *out = nullptr;
    auto* m = new icd2s_mlp();
    m->seed = seed;
    cudaError_t e = cudaSuccess;
    if ((e = dalloc(&m->master, kNPar)) != cudaSuccess || (e = dalloc(&m->mom, kNPar)) != cudaSuccess ||
        (e = dalloc(&m->vel, kNPar)) != cudaSuccess || (e = dmalloc(&m->Wb, 2 * kNPar)) != cudaSuccess) {
        free_mlp(m);
        return fail(ICD2S_ERR_OOM, "device allocation failed: %s", cudaGetErrorString(e));
    }
    // Glorot-uniform weights from Philox (counter (q, TAG_MLP_INIT << 24, 0, 0)), zero biases
    std::vector<float> W(kNPar, 0.f);
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    auto fill = [&](int off, int count, int fan_in, int fan_out) {
        const double bound = std::sqrt(6.0 / (double)(fan_in + fan_out));
        for (int i = 0; i < count; ++i) {
            const u32x4 v = philox10((uint32_t)(off + i), kTagMlpInit << 24, 0u, 0u, k0, k1);
            const double u = (double)v.v[0] * (1.0 / 4294967296.0);
            W[off + i] = (float)((2.0 * u - 1.0) * bound);
        }
    };
    fill(kOffW1, 384, 6, 64);
    fill(kOffW2, 4096, 64, 64);
    fill(kOffW3, 64, 64, 1);
    const int rc = mlp_upload(m, W.data());
    if (rc) { free_mlp(m); return rc; }
    *out = m;
    return ICD2S_OK;
}

int icd2s_mlp_destroy(icd2s_mlp* m)
{
    if (m) free_mlp(m);
    return ICD2S_OK;
}

int icd2s_mlp_set_weights(icd2s_mlp* m, const float* W_host)
{
    REQ(m && W_host, ICD2S_ERR_ARG, "NULL argument");
    for (int q = 0; q < kNPar; ++q) REQ(std::isfinite(W_host[q]), ICD2S_ERR_ARG, "weight %d is not finite", q);
    return mlp_upload(m, W_host);
}

int icd2s_mlp_get_weights(icd2s_mlp* m, float* master_host, float* bf16_host)
{
    REQ(m, ICD2S_ERR_ARG, "NULL network");
    CK(cudaDeviceSynchronize());
    if (master_host) CK(cudaMemcpy(master_host, m->master, sizeof(float) * kNPar, cudaMemcpyDeviceToHost));
    if (bf16_host) {
        std::vector<uint16_t> b(kNPar);
        CK(cudaMemcpy(b.data(), m->Wb, 2 * kNPar, cudaMemcpyDeviceToHost));
        for (int q = 0; q < kNPar; ++q) {
            const uint32_t bits = (uint32_t)b[q] << 16;
            std::memcpy(&bf16_host[q], &bits, 4);
        }
    }
    return ICD2S_OK;
}

int icd2s_mlp_score(icd2s_mlp* m, const float* F_dev, int64_t rows, float* score_dev, void* stream)
{
    REQ(m && (rows == 0 || (F_dev && score_dev)), ICD2S_ERR_ARG, "NULL argument");
    REQ(rows >= 0, ICD2S_ERR_ARG, "rows < 0");
    CK(launch_score(F_dev, rows, m->Wb, score_dev, S(stream)));
    return ICD2S_OK;
}

static int ensure_partial(icd2s_mlp* m, long long batch, cudaStream_t s)
{
    const size_t need = mlp_partial_floats(batch);
    if (need <= m->partial_cap) return ICD2S_OK;
    CK(cudaStreamSynchronize(s));
    if (m->partial) CK(cudaFree(m->partial));
    m->partial = nullptr;
    m->partial_cap = 0;
    CK(dalloc(&m->partial, need));
    m->partial_cap = need;
    return ICD2S_OK;
}

int icd2s_mlp_grad(icd2s_mlp* m, const float* F_dev, const uint8_t* y_dev, int64_t rows, float pos_weight,
                   float* grad_dev, float* loss_dev, void* stream)
{
    REQ(m && F_dev && y_dev, ICD2S_ERR_ARG, "NULL argument");
    REQ(rows >= 1 && rows <= ((int64_t)1 << 31) * 64, ICD2S_ERR_RANGE, "rows=%lld out of range", (long long)rows);
    REQ(std::isfinite(pos_weight) && pos_weight >= 0.f, ICD2S_ERR_ARG, "pos_weight must be finite and >= 0");
    cudaStream_t s = S(stream);
    int rc = ensure_partial(m, rows, s);
    if (rc) return rc;
    CK(launch_mlp_grad(F_dev, y_dev, rows, rows, 0u, 0u, 0u, m->Wb, pos_weight, m->partial, grad_dev, loss_dev,
                       nullptr, nullptr, nullptr, nullptr, 0, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, s, m->tensor_cores));
    return ICD2S_OK;
}

int icd2s_mlp_train(icd2s_mlp* m, const float* F_dev, const uint8_t* y_dev, int64_t rows,
                    const icd2s_train_params* tp, float* loss_host, void* stream)
{
    REQ(m && F_dev && y_dev && tp, ICD2S_ERR_ARG, "NULL argument");
    REQ(rows >= 1 && rows <= ((int64_t)1 << 31) * 64, ICD2S_ERR_RANGE, "rows=%lld out of range", (long long)rows);
    REQ(tp->steps >= 0 && tp->batch >= 1, ICD2S_ERR_ARG, "steps >= 0 and batch >= 1 required");
    REQ(std::isfinite(tp->lr) && tp->lr >= 0.f && tp->beta1 >= 0.f && tp->beta1 < 1.f && tp->beta2 >= 0.f &&
        tp->beta2 < 1.f && tp->eps > 0.f && std::isfinite(tp->pos_weight) && tp->pos_weight >= 0.f,
        ICD2S_ERR_ARG, "bad training parameters");
    if (tp->steps == 0) return ICD2S_OK;
    cudaStream_t s = S(stream);
    const long long batch = tp->batch < rows ? tp->batch : rows;
    int rc = ensure_partial(m, batch, s);
    if (rc) return rc;
    if (tp->steps > m->loss_cap) {
        CK(cudaStreamSynchronize(s));
        if (m->losses) CK(cudaFree(m->losses));
        m->losses = nullptr;
        m->loss_cap = 0;
        CK(dalloc(&m->losses, (size_t)tp->steps));
        m->loss_cap = tp->steps;
    }
    const uint32_t k0 = (uint32_t)(m->seed & 0xffffffffu), k1 = (uint32_t)(m->seed >> 32);
    for (int i = 0; i < tp->steps; ++i) {
        const int64_t t = m->adam_t + 1;
        const float bc1 = (float)(1.0 - std::pow((double)tp->beta1, (double)t));
        const float bc2 = (float)(1.0 - std::pow((double)tp->beta2, (double)t));
        CK(launch_mlp_grad(F_dev, y_dev, rows, tp->batch, (uint32_t)m->adam_t, k0, k1, m->Wb, tp->pos_weight,
                           m->partial, nullptr, m->losses + i, m->master, m->mom, m->vel, m->Wb, 1, tp->lr,
                           tp->beta1, tp->beta2, tp->eps, bc1, bc2, s, m->tensor_cores));
        m->adam_t = t;
    }
    if (loss_host) {
        CK(cudaMemcpyAsync(loss_host, m->losses, sizeof(float) * tp->steps, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return ICD2S_OK;
}

int icd2s_mlp_set_tensor_cores(icd2s_mlp* m, int32_t enable)
{
    REQ(m, ICD2S_ERR_ARG, "NULL network");
    REQ(enable == 0 || enable == 1, ICD2S_ERR_ARG, "enable must be 0 or 1");
    m->tensor_cores = enable != 0;
    return ICD2S_OK;
}

int icd2s_state_set_mlp(icd2s_state* st, icd2s_mlp* m)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    st->mlp = m;
    ++st->gen;  // the captured step holds the network's weights pointer
    return ICD2S_OK;
}

int icd2s_get_features(icd2s_state* st, float* F_host, float* score_host)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    REQ(st->have_features && (score_host == nullptr || st->have_scores), ICD2S_ERR_STATE,
        "no step has computed features%s yet", score_host ? " and scores" : "");
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    CK(cudaDeviceSynchronize());
    if (F_host)
        CK(cudaMemcpy2D(F_host, (size_t)n * 24, st->F, (size_t)ld * 24, (size_t)n * 24, R, cudaMemcpyDeviceToHost));
    if (score_host)
        CK(cudaMemcpy2D(score_host, (size_t)n * 4, st->score, (size_t)ld * 4, (size_t)n * 4, R,
                        cudaMemcpyDeviceToHost));
    return ICD2S_OK;
}

int icd2s_get_hits(icd2s_state* st, int32_t* H_host)
{
    REQ(st && H_host, ICD2S_ERR_ARG, "NULL argument");
    const int n = st->q->n, ld = st->q->ld, R = st->R;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy2D(H_host, (size_t)n * 4, st->H, (size_t)ld * 4, (size_t)n * 4, R, cudaMemcpyDeviceToHost));
    return ICD2S_OK;
}

int icd2s_log_enable(icd2s_state* st, int32_t capacity)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    REQ(capacity >= 0, ICD2S_ERR_ARG, "capacity < 0");
    const int n = st->q->n;
    REQ((int64_t)capacity * n <= ((int64_t)1 << 31), ICD2S_ERR_RANGE, "capacity * n above 2^31 rows");
    CK(cudaDeviceSynchronize());
    void* ptrs[] = {st->LF, st->LY, st->lrep, st->prev_x, st->log_ctl};
    for (void* p : ptrs)
        if (p) CK(cudaFree(p));
    st->LF = nullptr; st->LY = nullptr; st->lrep = nullptr; st->prev_x = nullptr; st->log_ctl = nullptr;
    st->log_cap = 0;
    ++st->gen;
    if (capacity == 0) return ICD2S_OK;
    CK(dalloc(&st->LF, (size_t)capacity * n * 6));
    CK(dalloc(&st->LY, (size_t)capacity * n));
    CK(dalloc(&st->lrep, (size_t)capacity));
    CK(dalloc(&st->prev_x, (size_t)st->q->ld));
    CK(dalloc(&st->log_ctl, 2));
    const int32_t ctl[2] = {0, capacity};
    CK(cudaMemcpy(st->log_ctl, ctl, 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(st->prev_x, st->best_x, (size_t)st->q->ld, cudaMemcpyDeviceToDevice));
    st->log_cap = capacity;
    return ICD2S_OK;
}

int icd2s_log_info(icd2s_state* st, int32_t* entries, int32_t* capacity)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    int32_t ctl[2] = {0, 0};
    if (st->log_cap > 0) {
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(ctl, st->log_ctl, 8, cudaMemcpyDeviceToHost));
    }
    if (entries) *entries = ctl[0];
    if (capacity) *capacity = st->log_cap;
    return ICD2S_OK;
}

int icd2s_log_copy(icd2s_state* st, float* F_out, uint8_t* y_out, int32_t* replica_out, int32_t out_is_device,
                   void* stream)
{
    REQ(st, ICD2S_ERR_ARG, "NULL state");
    REQ(st->log_cap > 0, ICD2S_ERR_STATE, "logging is off (icd2s_log_enable)");
    cudaStream_t s = S(stream);
    int32_t ctl[2] = {0, 0};
    CK(cudaMemcpyAsync(ctl, st->log_ctl, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const size_t cnt = (size_t)(ctl[0] < st->log_cap ? ctl[0] : st->log_cap), n = (size_t)st->q->n;
    const cudaMemcpyKind k = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cnt > 0) {
        if (F_out) CK(cudaMemcpyAsync(F_out, st->LF, cnt * n * 24, k, s));
        if (y_out) CK(cudaMemcpyAsync(y_out, st->LY, cnt * n, k, s));
        if (replica_out) CK(cudaMemcpyAsync(replica_out, st->lrep, cnt * 4, k, s));
    }
    CK(cudaStreamSynchronize(s));
    return ICD2S_OK;
}

}  // extern "C"
