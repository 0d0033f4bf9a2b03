// Launcher of the fused CGS2 / Givens / normalisation kernel (k_cgs_fused):
// one cooperative launch whose blocks each keep a contiguous chunk of w in
// shared memory, or `false` when the chunks do not fit (the caller then uses
// the three separate kernels).
#include "ctx.h"
#include "fused.cuh"
#include "step.cuh"

namespace f3r {

namespace {

template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                        Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// 2 blocks of 512 threads per SM when the chunk fits, else 1; every block of
// the grid must be resident at once (the launch is cooperative)
template <class K> FusedPlan fused_plan(const Ctx &c, K kern, int tsize) {
    FusedPlan p;
    for (int bps = 2; bps >= 1; --bps) {
        const int G = c.nsm * bps;
        const int per = ceil_div(c.n, G);
        const int chunk = ceil_div(per, kFusedChunkAlign) * kFusedChunkAlign;
        const int smem = chunk * tsize;
        if (smem > 200 * 1024) continue;
        if (!ensure_dyn_smem((const void *)kern, smem)) continue;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kFusedThreads, smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nb < bps) continue;
        p.G = ceil_div(c.n, chunk);
        p.chunk = chunk;
        p.smem = smem;
        return p;
    }
    return p;
}

template <class T> LevelDev<T> levdev_inner(Ctx &c, int d) {
    LevelDev<T> L;
    L.n = c.n;
    L.ld = c.ld;
    L.m = c.L[d].m;
    L.depth = d;
    L.rtol = (d >= 1 && d == c.prm.nlevels - 1) ? c.prm.inner_rtol : 0.0f;
    L.V = (T *)c.L[d].V;
    L.Z = (T *)c.L[d].Z;
    L.w = (T *)c.L[d].w;
    L.scal = (T *)c.L[d].scal;
    L.flags = c.flags;
    L.jptr = nullptr;
    L.vround = vround_of(c, d);
    return L;
}

int want_sigma_of(const Ctx &c, int d) {
    const bool rich_half = c.prm.rich_m > 0 && (c.prm.rich_v_prec == F3R_F16 || c.prm.rich_v_prec == F3R_BF16);
    return (c.L[d].child == CHILD_R && rich_half && c.prm.scale_cast) ? 1 : 0;
}

// plan_only: size the launch of level d into c.fplan[d] (at set-up, outside
// any stream capture); else launch with that plan
template <class T, class TC, int CHILD, int MAXD>
bool fused_go(Ctx &c, int d, int j, bool last, bool do_norm, cudaStream_t s, bool plan_only) {
    auto kern = k_cgs_fused<T, TC, CHILD, MAXD>;
    if (plan_only) {
        c.fplan[d] = fused_plan(c, kern, (int)sizeof(T));
        return c.fplan[d].G > 0;
    }
    const FusedPlan p = c.fplan[d];
    if (p.G == 0) return false;
    ChildOut<TC> co{};
    if (CHILD == CHILD_F) {
        co.x = (TC *)c.L[d + 1].V;
        co.dsc = nullptr;
        co.cscal = c.L[d + 1].scal;
        co.cm = c.L[d + 1].m;
        co.cdepth = d + 1;
        co.want_sigma = want_sigma_of(c, d + 1);
    } else if (CHILD == CHILD_R) {
        co.x = (TC *)c.rin;
    }
    FusedScratch<T> fs{(T *)c.partials, c.coop, c.err, p.chunk, c.hpart_G[d] ? (const T *)c.hpart : nullptr, c.hpart_G[d]};
    GridRed<TC> grc{(TC *)c.partials, c.ticket, kMaxDots};
    return launch_coop(kern, dim3(p.G), dim3(kFusedThreads), p.smem, s, levdev_inner<T>(c, d), j,
                       c.prm.cgs_passes, last ? 1 : 0, want_sigma_of(c, d), do_norm ? 1 : 0, co, fs, grc) ==
           cudaSuccess;
}

template <class T, class TC, int CHILD>
bool fused_md(Ctx &c, int d, int j, bool last, bool do_norm, cudaStream_t s, bool plan_only) {
    const int md = maxd_bucket(c.L[d].m);
    if (md == 4) return fused_go<T, TC, CHILD, 4>(c, d, j, last, do_norm, s, plan_only);
    if (md == 8) return fused_go<T, TC, CHILD, 8>(c, d, j, last, do_norm, s, plan_only);
    return fused_go<T, TC, CHILD, 16>(c, d, j, last, do_norm, s, plan_only);
}

bool fused_dispatch(Ctx &c, int d, int j, bool last, bool do_norm, cudaStream_t s, bool plan_only) {
    const bool t64 = c.L[d].v_prec == F3R_F64;
    const int ch = c.L[d].child;
    if (ch == CHILD_F) {
        const bool c64 = c.L[d + 1].v_prec == F3R_F64;
        if (t64 && c64) return fused_md<double, double, CHILD_F>(c, d, j, last, do_norm, s, plan_only);
        if (t64) return fused_md<double, float, CHILD_F>(c, d, j, last, do_norm, s, plan_only);
        if (c64) return fused_md<float, double, CHILD_F>(c, d, j, last, do_norm, s, plan_only);
        return fused_md<float, float, CHILD_F>(c, d, j, last, do_norm, s, plan_only);
    }
    if (ch == CHILD_R) {
        switch (c.prm.rich_v_prec) {
            case F3R_F64: return fused_md<double, double, CHILD_R>(c, d, j, last, do_norm, s, plan_only);
            case F3R_F32:
                return t64 ? fused_md<double, float, CHILD_R>(c, d, j, last, do_norm, s, plan_only)
                           : fused_md<float, float, CHILD_R>(c, d, j, last, do_norm, s, plan_only);
            case F3R_F16:
                return t64 ? fused_md<double, h16, CHILD_R>(c, d, j, last, do_norm, s, plan_only)
                           : fused_md<float, h16, CHILD_R>(c, d, j, last, do_norm, s, plan_only);
            default:
                return t64 ? fused_md<double, b16, CHILD_R>(c, d, j, last, do_norm, s, plan_only)
                           : fused_md<float, b16, CHILD_R>(c, d, j, last, do_norm, s, plan_only);
        }
    }
    return t64 ? fused_md<double, double, CHILD_M>(c, d, j, last, do_norm, s, plan_only)
               : fused_md<float, float, CHILD_M>(c, d, j, last, do_norm, s, plan_only);
}

template <class TC, int CHILD> bool outer_go(Ctx &c, cudaStream_t s, bool plan_only) {
    auto kern = k_outer_cgs_fused<TC, CHILD>;
    if (plan_only) {
        c.fplan[0] = fused_plan(c, kern, (int)sizeof(double));
        return c.fplan[0].G > 0;
    }
    const FusedPlan p = c.fplan[0];
    if (p.G == 0) return false;
    ChildOut<TC> co{};
    if (CHILD == CHILD_F) {
        co.x = (TC *)c.L[1].V;
        co.dsc = c.prm.diag_scale ? c.dsc : nullptr;
        co.cscal = c.L[1].scal;
        co.cm = c.L[1].m;
        co.cdepth = 1;
        co.want_sigma = want_sigma_of(c, 1);
    }
    LevelDev<double> L = levdev_inner<double>(c, 0);
    L.jptr = c.jdev;
    FusedScratch<double> fs{(double *)c.partials, c.coop, c.err, p.chunk};
    GridRed<TC> grc{(TC *)c.partials, c.ticket, kMaxDots};
    return launch_coop(kern, dim3(p.G), dim3(kFusedThreads), p.smem, s, L, c.prm.cgs_passes, co, fs, grc) ==
           cudaSuccess;
}

// the outer level's child: an FGMRES level (fp32 or fp64 vectors) or M; a
// Richardson child keeps the separate kernels
bool outer_dispatch(Ctx &c, cudaStream_t s, bool plan_only) {
    const int ch = c.L[0].child;
    if (ch == CHILD_F)
        return c.L[1].v_prec == F3R_F64 ? outer_go<double, CHILD_F>(c, s, plan_only)
                                        : outer_go<float, CHILD_F>(c, s, plan_only);
    if (ch == CHILD_M) return outer_go<double, CHILD_M>(c, s, plan_only);
    return false;
}

// ---------------------------------------------------------------- whole step
bool step_eligible(const Ctx &c, int d) {
    const f3r_params &p = c.prm;
    return p.fuse_cgs && c.coop && d >= 1 && d == p.nlevels - 1 && c.L[d].child == CHILD_R && c.L[d].m <= kMaxInnerM &&
           c.L[d].v_prec == F3R_F32 && c.L[d].a_prec == F3R_F16 && p.rich_m == 2 && p.rich_v_prec == F3R_F16 &&
           p.rich_a_prec == F3R_F16 && p.m_prec == F3R_F16 && p.precond == F3R_PC_JACOBI && c.a16;
}

template <int S, int MAXD> bool step_go(Ctx &c, int d, int j, bool last, cudaStream_t s, bool plan_only) {
    auto kern = k_f3_step<S, MAXD>;
    if (plan_only) {
        // the first (blocks per SM, ring depth S) that fits, more blocks first
        StepPlan p = c.stplan;
        if (p.G > 0) return true;
        const StagePlan sp = plan_stage(c, sizeof(h16), c.L[d].m, sizeof(float));
        if (sp.S == 0) return false;
        const int ntiles = ceil_div(c.nslices, kTileSlices);
        for (int bps = c.stplan_bps; bps >= c.stplan_bps; --bps) {
            const int G = std::min(c.nsm * bps, ntiles);
            const int per = ceil_div(ntiles, G);
            const long long smem = kBarBytes + (long long)S * sp.stage_bytes + (long long)per * kTileRows * 4;
            if (smem > 220 * 1024) continue;
            if (!ensure_dyn_smem((const void *)kern, (int)smem)) {
                cudaGetLastError();
                continue;
            }
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kStagedThreads, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (nb < bps) continue;
            p.G = G;
            p.S = S;
            p.stage_bytes = sp.stage_bytes;
            p.smem = (int)smem;
            break;
        }
        c.stplan = p;
        return p.G > 0;
    }
    const StepPlan p = c.stplan;
    if (p.G == 0 || p.S != S) return false;
    StepArgs a;
    a.A = sell_of(c);
    a.a16 = c.a16;
    a.rs = c.prm.row_scale ? c.rs : nullptr;
    a.v16 = (const h16 *)c.rin;
    a.m16 = (const h16 *)c.mvec;
    a.zout = (float *)c.L[d].Z + (size_t)j * c.ld;
    a.omega = (const float *)c.omega;
    a.counters = c.counters;
    a.v16_next = (h16 *)c.rin;
    a.stage_bytes = p.stage_bytes;
    a.err = c.err;
    a.bar = c.coop;
    a.part = (float *)c.partials;
    const int do_norm = (j < c.L[d].m - 1) ? 1 : 0;
    return launch_coop(kern, dim3(p.G), dim3(kStagedThreads), p.smem, s, a, levdev_inner<float>(c, d), j, last ? 1 : 0,
                       want_sigma_of(c, d), do_norm) == cudaSuccess;
}

bool step_dispatch(Ctx &c, int d, int j, bool last, cudaStream_t s, bool plan_only, int S_try = 0) {
    const int md = maxd_bucket(c.L[d].m);
    const int S = plan_only ? S_try : c.stplan.S;
    if (S == 3) {
        if (md == 4) return step_go<3, 4>(c, d, j, last, s, plan_only);
        if (md == 8) return step_go<3, 8>(c, d, j, last, s, plan_only);
        return step_go<3, 16>(c, d, j, last, s, plan_only);
    }
    if (S == 2) {
        if (md == 4) return step_go<2, 4>(c, d, j, last, s, plan_only);
        if (md == 8) return step_go<2, 8>(c, d, j, last, s, plan_only);
        return step_go<2, 16>(c, d, j, last, s, plan_only);
    }
    return false;
}

}  // namespace

bool launch_f3_step(Ctx &c, int d, int j, bool last, bool update, cudaStream_t s) {
    if (update || c.stplan.G == 0 || d != c.prm.nlevels - 1) return false;
    prof_begin(c, PK_STEP, d, s);
    step_dispatch(c, d, j, last, s, false);
    prof_end(c, s);
    c.launches++;
    return true;
}

void plan_cgs_fused(Ctx &c) {
    for (int d = 0; d < 4; ++d) c.fplan[d] = FusedPlan{};
    if (!c.prm.fuse_cgs || !c.coop) return;
    outer_dispatch(c, nullptr, true);
    for (int d = 1; d < c.prm.nlevels; ++d)
        if (c.L[d].m <= kMaxInnerM) fused_dispatch(c, d, 0, false, false, nullptr, true);
    c.stplan = StepPlan{};
    const int d = c.prm.nlevels - 1;
    if (!c.prm.fuse_step || !step_eligible(c, d)) return;
    for (int bps = 4; bps >= 1 && c.stplan.G == 0; --bps) {
        c.stplan_bps = bps;
        for (int S = 3; S >= 2 && c.stplan.G == 0; --S) step_dispatch(c, d, 0, false, nullptr, true, S);
    }
}

bool launch_outer_cgs_fused(Ctx &c, cudaStream_t s) {
    if (c.fplan[0].G == 0) return false;
    prof_begin(c, PK_OUTER_CGS, 0, s);
    outer_dispatch(c, s, false);
    prof_end(c, s);
    c.launches++;
    return true;
}

bool launch_cgs_fused(Ctx &c, int d, int j, bool last, bool do_norm, cudaStream_t s) {
    if (d < 1 || d > 3 || c.fplan[d].G == 0) return false;
    prof_begin(c, PK_CGS_FUSED, d, s);
    fused_dispatch(c, d, j, last, do_norm, s, false);
    prof_end(c, s);
    c.launches++;
    return true;
}

}  // namespace f3r
