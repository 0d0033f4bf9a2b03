// Host-side state of one solver context and the launchers shared by the
// translation units of libf3r.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <vector>

#include "common.cuh"
#include "stage.cuh"

namespace f3r {

struct LearnedState;

struct LevelHost {
    int m = 0, a_prec = 0, v_prec = 0, child = 2;
    void *V = nullptr, *Z = nullptr, *w = nullptr, *scal = nullptr;
};

// What the host reads back after every outer iteration (pinned memory).
struct Readback {
    double est;       // |g_{j+1}| / ||b||
    double rel;       // true relative residual at a cycle start
    double nb;        // ||b||
    int err;          // device error word
    int flags[16];    // copy of all levels' flags
    unsigned long long counters[4];
};

// Where an FGMRES level writes its result z.
struct OutSlot {
    void *ptr = nullptr;    // vector of type out_prec
    int prec = F3R_F32;
    bool dscale = false;    // multiply by D^-1/2 (return to the outer level)
};

// Kernel timing slots (kind * 4 + level) for the event profiler.
enum {
    PK_SPMV_DOTS = 0, PK_CGS_PASS, PK_CGS_FINAL, PK_NORMALIZE, PK_COMBINE, PK_START, PK_M, PK_RICH2,
    PK_RICH_STEP, PK_RICH_UPD, PK_OUTER_SPMV, PK_OUTER_CGS, PK_OUTER_OTHER, PK_SPMV, PK_CGS_FUSED, PK_STEP, PK_KINDS
};
constexpr int kProfSlots = PK_KINDS * 4;

struct ProfRec {
    int slot;
    cudaEvent_t a, b;
};

// Launch shape of the fused CGS2 / normalisation kernel of one level
// (G == 0: not fused).
struct FusedPlan {
    int G = 0, chunk = 0, smem = 0;
};

// Launch shape of the whole-iteration kernel of the innermost level (G == 0: off).
struct StepPlan {
    int G = 0, S = 0, stage_bytes = 0, smem = 0;
};

struct Ctx {
    int dev = 0, nsm = 0;
    cudaStream_t zstream = nullptr;  // the context's stream (zero-fills of allocations)
    f3r_params prm{};
    int n = 0;
    long long nnz = 0;
    int ld = 0;            // stride between vectors of a basis
    // sliced ELLPACK (slices of 32 rows, column-major inside a slice)
    int nslices = 0;
    int wmax = 0;              // widest slice (entries per row)
    long long nsell = 0;
    int *sptr = nullptr, *col = nullptr, *rowptr = nullptr;
    // windowed tiles (stage.cuh): 16-bit window index per SELL entry and one
    // record of x runs per 256-row tile; win = every tile fits its window
    uint16_t *lcol = nullptr;
    int *wrec = nullptr;
    bool win = false;
    int win_max = 0;            // largest window of any tile (entries)
    double *a64 = nullptr;      // original A
    double *ah64 = nullptr;     // scaled A^ in fp64
    float *a32 = nullptr;       // A^ in fp32
    h16 *a16 = nullptr;         // A^ / s in fp16
    b16 *abf = nullptr;         // A^ / s in bf16
    float *rs = nullptr;        // power-of-two row scales s (row_scale = 1)
    double *dsc = nullptr;      // D^-1/2
    void *mvec = nullptr;       // M in m_prec
    bool m_unit = false;        // every stored entry of M is exactly 1 (M = I)
    // approximate inverse M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1) (precond = F3R_PC_AINV)
    h16 *ainv_l = nullptr, *ainv_u = nullptr;  // L Dt^-1 and Dt^-1 U on the SELL pattern (fp16)
    h16 *ainv_dinv = nullptr;                  // Dt^-1 (fp16)
    float *ainv_t = nullptr, *ainv_m = nullptr;  // Dt^-1 (I - L Dt^-1) r and M r (fp32)
    LevelHost L[4];
    // Richardson
    void *rin = nullptr, *rz[2] = {nullptr, nullptr}, *rr = nullptr;
    void *omega = nullptr, *wcur = nullptr;
    unsigned long long *counters = nullptr;
    long long *c_ntr_base = nullptr;
    long long c_ntr = 1;
    double omega_host[kMaxRich];
    int calls_per_outer = 0;
    // reductions and flags
    void *partials = nullptr;
    unsigned *ticket = nullptr;
    unsigned *coop = nullptr;   // grid-barrier counters of cooperative launches (zero between launches)
    void *hpart = nullptr;      // [l][block] totals of hA left by the SpMV + dots for the fused CGS2
    int hpart_G[4] = {0, 0, 0, 0};  // blocks of that SpMV per level (0: it reduced hA itself)
    FusedPlan fplan[4];
    StepPlan stplan;
    int stplan_bps = 0;         // blocks per SM the step plan is being tried with
    int G = 1, Gs = 1, G1 = 1, Gv = 1;  // grids: elementwise, SpMV, outer CGS, streaming vector kernels
    int *flags = nullptr;       // 4 ints per level
    int *err = nullptr;         // device error word (bounded waits that gave up)
    bool staged = true;         // stage SELL slices through shared memory
    int *jdev = nullptr;
    void *zst = nullptr;        // the outer level's preconditioner output (fp64)
    void *apply_misc = nullptr; // scalars of a stand-alone Richardson call
    double *bdev = nullptr, *xdev = nullptr;
    Readback *rb = nullptr;     // pinned
    double *hostval = nullptr;  // pinned scratch
    std::map<long long, cudaGraphExec_t> graphs;
    long long launches = 0, graph_launches = 0;
    long long launches_per_graph_iter = 0;
    long long bytes = 0;
    std::vector<void *> allocs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // event profiler: when on, every launch is bracketed by two events on its stream
    bool prof = false;
    std::vector<ProfRec> prec;
    size_t prec_used = 0;
    double prof_ms[kProfSlots] = {};
    long long prof_cnt[kProfSlots] = {};
    LearnedState *learned = nullptr;  // learned preconditioner (precond = F3R_PC_LEARNED)
    void *krylov = nullptr;           // CG / BiCGStab comparator state (krylov.cu)
};

inline void prof_begin(Ctx &c, int kind, int level, cudaStream_t s) {
    if (!c.prof) return;
    if (c.prec_used == c.prec.size()) {
        ProfRec r;
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
        c.prec.push_back(r);
    }
    ProfRec &r = c.prec[c.prec_used];
    r.slot = kind * 4 + (level & 3);
    cudaEventRecord(r.a, s);
}
inline void prof_end(Ctx &c, cudaStream_t s) {
    if (!c.prof) return;
    cudaEventRecord(c.prec[c.prec_used].b, s);
    c.prec_used++;
}
// after a synchronisation: fold the recorded pairs into the per-slot totals
inline void prof_collect(Ctx &c) {
    for (size_t i = 0; i < c.prec_used; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c.prec[i].a, c.prec[i].b) == cudaSuccess) {
            c.prof_ms[c.prec[i].slot] += ms;
            c.prof_cnt[c.prec[i].slot] += 1;
        }
    }
    c.prec_used = 0;
}

inline Sell sell_of(const Ctx &c) { return Sell{c.n, c.nslices, c.sptr, c.col}; }

// setup.cu
f3r_status build_matrix(Ctx &c, const int *rowptr_d, const int *colidx_d, const double *val_d, cudaStream_t s);
// window.cu: windowed tiles of the SELL matrix (sets c.win); the Window a
// kernel gathering x of xsize bytes (n entries) takes (empty when not windowed)
f3r_status build_window(Ctx &c, cudaStream_t s);
Window window_of(const Ctx &c, int xsize, int n);
f3r_status export_array(Ctx &c, int which, void *out, cudaStream_t s);

// launch_levels.cu
void launch_level_start(Ctx &c, int d, const void *x, cudaStream_t s);
void launch_normalize(Ctx &c, int d, bool from_w, int dst, cudaStream_t s);
void launch_spmv_dots(Ctx &c, int d, int j, cudaStream_t s);
void launch_cgs_pass(Ctx &c, int d, int j, cudaStream_t s);
void launch_cgs_final(Ctx &c, int d, int j, bool last, cudaStream_t s);
// launch_fused.cu
void plan_cgs_fused(Ctx &c);
bool launch_cgs_fused(Ctx &c, int d, int j, bool last, bool do_norm, cudaStream_t s);
bool launch_outer_cgs_fused(Ctx &c, cudaStream_t s);
bool launch_f3_step(Ctx &c, int d, int j, bool last, bool update, cudaStream_t s);
void launch_combine(Ctx &c, int d, const OutSlot &o, cudaStream_t s);
// w = A_l Z[j], CGS2 and the Givens step of an inner level with m > kMaxInnerM
void launch_long_step(Ctx &c, int d, int j, bool last, cudaStream_t s);
// vround: the output is a level's stored Z[j] rounded to 16 bits (vround_of)
void launch_M(Ctx &c, int d, int j, const void *in, void *out, int check_depth, bool use_j, cudaStream_t s,
              int vround = 0);
// 1 / 2 when FGMRES level d stores its vectors in fp16 / bf16 (Table 4's fp16 levels), else 0
inline int vround_of(const Ctx &c, int d) {
    if (d < 1) return 0;
    const int v = c.prm.v_prec[d];
    return v == F3R_F16 ? 1 : (v == F3R_BF16 ? 2 : 0);
}
// bytes per element of level d's vector arrays (16-bit levels keep fp32 arrays)
inline int level_vec_bytes(const Ctx &c, int d) { return c.prm.v_prec[d] == F3R_F64 ? 8 : 4; }
void launch_outer_residual(Ctx &c, const double *b, const double *x, bool compute_nb, cudaStream_t s);
bool launch_outer_step(Ctx &c, cudaStream_t s);
void launch_outer_finish(Ctx &c, double *x, cudaStream_t s);
void launch_advance(Ctx &c, long long inc, cudaStream_t s);
f3r_status launch_spmv(Ctx &c, int p, int vp, const void *x, void *y, cudaStream_t s);

// launch_rich.cu
void launch_rich_call(Ctx &c, bool update, int pos, void *out, const void *par_misc, cudaStream_t s);
void launch_rich_prep(Ctx &c, const void *x, cudaStream_t s);

// learned.cu
f3r_status learned_enable(Ctx &c, const float *theta, bool train);
void learned_forward(Ctx &c, const float *r, float *z, bool train, cudaStream_t s);
f3r_status learned_loss_grad(Ctx &c, const float *R, const float *E, int P, cudaStream_t s);
void learned_adam(Ctx &c, float lr, cudaStream_t s);
void learned_rich_call(Ctx &c, bool update, int pos, void *out, const void *par_misc, cudaStream_t s);
void learned_free(Ctx &c);

// ainv.cu: Richardson call with the approximate inverse as M
void ainv_rich_call(Ctx &c, bool update, int pos, void *out, const void *par_misc, cudaStream_t s);
f3r_status learned_set_loss(Ctx &c, int kind);
int learned_loss_kind(const Ctx &c);
float *learned_theta(Ctx &c);
float *learned_grad(Ctx &c);
float *learned_loss(Ctx &c);

// krylov.cu: CG (method 1) / BiCGStab (method 2) on the original fp64 A
f3r_status krylov_solve(Ctx &c, cudaStream_t s, int method, const double *b, double *x, int max_iters,
                        f3r_stats *stats);
void krylov_free(Ctx &c);

// sizes
int prec_bytes(int p);

// Shared-memory staging plan of one SELL kernel: ring depth S, bytes per
// stage, dynamic shared memory per block and the grid (resident blocks).
struct StagePlan {
    int S = 0, stage_bytes = 0, smem = 0;
};
// xsize > 0: a windowed kernel gathering x of xsize bytes (sized for the
// widest window; only meaningful when c.win)
StagePlan plan_stage(const Ctx &c, int asize, int n_extra, int esize, int xsize = 0);
// stream-ordered device memory from the per-device pool (mem.cu)
void *pool_alloc(int dev, size_t bytes, cudaStream_t s);
// Raise the dynamic shared memory limit of a kernel to at least `bytes`,
// never lowering it: contexts of different sizes in one process share the
// kernel, and a plan made by one must still launch after another's (mem.cu)
bool ensure_dyn_smem(const void *kern, int bytes);
void pool_free(void *p, cudaStream_t s);
int maxd_bucket(int m);

}  // namespace f3r
