// Launchers of the FGMRES-level kernels, dispatching on the precisions of
// each level (Table 1).
#include "ctx.h"
#include "kernels.cuh"
#include "staged.cuh"

namespace f3r {

template <class T> static LevelDev<T> levdev(Ctx &c, int d) {
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
    L.jptr = (d == 0) ? c.jdev : nullptr;
    L.vround = vround_of(c, d);
    return L;
}

template <class T> static GridRed<T> gred(Ctx &c, int stride) {
    return GridRed<T>{(T *)c.partials, c.ticket, stride};
}

static bool rich_half(const Ctx &c) {
    return c.prm.rich_m > 0 && (c.prm.rich_v_prec == F3R_F16 || c.prm.rich_v_prec == F3R_BF16);
}

// the level below d wants the 16-bit cast scale of V[j+1]
static int want_sigma(const Ctx &c, int d) {
    return (c.L[d].child == CHILD_R && rich_half(c) && c.prm.scale_cast) ? 1 : 0;
}

// ------------------------------------------------------------------ start
template <class T>
__global__ void __launch_bounds__(kBlock) k_level_start(const T *x, LevelDev<T> C, int want_sig, GridRed<T> gr) {
    pdl_enter();
    T acc[2] = {(T)0, (T)0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C.n; i += gridDim.x * blockDim.x) {
        const T v = x[i];
        C.V[i] = v;
        acc[0] = fma_rn(v, v, acc[0]);
        acc[1] = fmax(acc[1], fabs(v));
    }
    grid_reduce<T, 2>(acc, 1, true, gr, [&](T *res) {
        T *ms = C.misc();
        int *cf = C.fl();
        const T beta = sqrt_rn(res[0]);
        cf[IF_KDIM] = 0;
        cf[IF_NONFINITE] = isfinite(beta) ? 0 : 1;
        const bool run = (beta > (T)0) && isfinite(beta);
        cf[IF_STOP] = run ? 0 : 1;
        ms[MS_BETA] = beta;
        if (run) {
            ms[MS_INV] = div_rn((T)1, beta);
            C.g()[0] = beta;
            const T sg = want_sig ? pow2_scale_for(mul_rn(res[1], ms[MS_INV])) : (T)1;
            ms[MS_SIGMA] = sg;
            ms[MS_INV_SIGMA] = div_rn((T)1, sg);
        }
    });
}

void launch_level_start(Ctx &c, int d, const void *x, cudaStream_t s) {
    prof_begin(c, PK_START, d, s);
    if (c.L[d].v_prec == F3R_F64)
        launch_pdl(k_level_start<double>, dim3(c.G), dim3(kBlock), 0, s, (const double *)x, levdev<double>(c, d), want_sigma(c, d),
                                                      gred<double>(c, kMaxDots));
    else
        launch_pdl(k_level_start<float>, dim3(c.G), dim3(kBlock), 0, s, (const float *)x, levdev<float>(c, d), want_sigma(c, d),
                                                     gred<float>(c, kMaxDots));
    prof_end(c, s);
    c.launches++;
}

// -------------------------------------------------------------- normalise
template <class T, class TC, int CHILD>
static void norm_go(Ctx &c, int d, bool from_w, int dst, cudaStream_t s) {
    LevelDev<T> L = levdev<T>(c, d);
    ChildOut<TC> co{};
    if (CHILD == CHILD_F) {
        co.x = (TC *)c.L[d + 1].V;
        co.dsc = (d == 0 && c.prm.diag_scale) ? c.dsc : nullptr;
        co.cscal = c.L[d + 1].scal;
        co.cm = c.L[d + 1].m;
        co.cdepth = d + 1;
        co.want_sigma = want_sigma(c, d + 1);
    } else if (CHILD == CHILD_R) {
        co.x = (TC *)c.rin;
    }
    const T *src = from_w ? L.w : L.V;  // at a level start V[0] is normalised in place
    // V[0] of the outer level is addressed through j (= 0 at a cycle start)
    prof_begin(c, PK_NORMALIZE, d, s);
    launch_pdl(k_normalize<T, TC, CHILD>, dim3(c.Gv), dim3(kVecBlock), 0, s, L, src, dst, d, co, gred<T>(c, kMaxDots));
    prof_end(c, s);
    c.launches++;
}

void launch_normalize(Ctx &c, int d, bool from_w, int dst, cudaStream_t s) {
    const bool t64 = c.L[d].v_prec == F3R_F64;
    const int ch = c.L[d].child;
    if (ch == CHILD_F) {
        const bool c64 = c.L[d + 1].v_prec == F3R_F64;
        if (t64 && c64) norm_go<double, double, CHILD_F>(c, d, from_w, dst, s);
        else if (t64) norm_go<double, float, CHILD_F>(c, d, from_w, dst, s);
        else if (c64) norm_go<float, double, CHILD_F>(c, d, from_w, dst, s);
        else norm_go<float, float, CHILD_F>(c, d, from_w, dst, s);
    } else if (ch == CHILD_R) {
        switch (c.prm.rich_v_prec) {
            case F3R_F64: norm_go<double, double, CHILD_R>(c, d, from_w, dst, s); break;
            case F3R_F32:
                if (t64) norm_go<double, float, CHILD_R>(c, d, from_w, dst, s);
                else norm_go<float, float, CHILD_R>(c, d, from_w, dst, s);
                break;
            case F3R_F16:
                if (t64) norm_go<double, h16, CHILD_R>(c, d, from_w, dst, s);
                else norm_go<float, h16, CHILD_R>(c, d, from_w, dst, s);
                break;
            default:
                if (t64) norm_go<double, b16, CHILD_R>(c, d, from_w, dst, s);
                else norm_go<float, b16, CHILD_R>(c, d, from_w, dst, s);
                break;
        }
    } else {
        if (t64) norm_go<double, double, CHILD_M>(c, d, from_w, dst, s);
        else norm_go<float, float, CHILD_M>(c, d, from_w, dst, s);
    }
}

// ------------------------------------------------------------ SpMV + dots
// grid of a staged kernel: the blocks that fit on the SMs at once (<= 4 per SM)
template <class K> static int staged_grid(Ctx &c, K kern, int smem, int work_blocks) {
    ensure_dyn_smem((const void *)kern, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kStagedThreads, smem);
    nb = std::max(1, std::min(nb, 8));
    return std::max(1, std::min(c.nsm * nb, work_blocks));
}

template <class TA, class T, int S, int MAXD, bool WIN>
static void spmv_dots_st_go(Ctx &c, int d, int j, const TA *val, const float *rs, const StagePlan &pl,
                            cudaStream_t s) {
    auto kern = k_spmv_dots_st<TA, T, S, MAXD, WIN>;
    const int g = staged_grid(c, kern, pl.smem, ceil_div(c.nslices, kTileSlices));
    // block totals of hA for the fused CGS2 launch that follows, when it will run
    const bool defer = d >= 1 && d <= 3 && c.fplan[d].G > 0;
    c.hpart_G[d] = defer ? g : 0;
    launch_pdl(kern, dim3(g), dim3(kStagedThreads), pl.smem, s, sell_of(c), val, rs, levdev<T>(c, d), j, gred<T>(c, kMaxDots),
                                    StageCfg{pl.stage_bytes, c.err}, defer ? (T *)c.hpart : (T *)nullptr,
                                    WIN ? window_of(c, sizeof(T), c.n) : Window());
}

template <class TA, class T, bool WIN>
static bool spmv_dots_plan_go(Ctx &c, int d, int j, const TA *val, const float *rs, const StagePlan &pl,
                              cudaStream_t s) {
    const int md = maxd_bucket(c.L[d].m);
    if constexpr (WIN) {
        if (pl.S == 4) {
            if (md == 4) spmv_dots_st_go<TA, T, 4, 4, WIN>(c, d, j, val, rs, pl, s);
            else if (md == 8) spmv_dots_st_go<TA, T, 4, 8, WIN>(c, d, j, val, rs, pl, s);
            else spmv_dots_st_go<TA, T, 4, 16, WIN>(c, d, j, val, rs, pl, s);
            return true;
        }
    }
    if (pl.S == 3) {
        if (md == 4) spmv_dots_st_go<TA, T, 3, 4, WIN>(c, d, j, val, rs, pl, s);
        else if (md == 8) spmv_dots_st_go<TA, T, 3, 8, WIN>(c, d, j, val, rs, pl, s);
        else spmv_dots_st_go<TA, T, 3, 16, WIN>(c, d, j, val, rs, pl, s);
        return true;
    }
    if (pl.S == 2) {
        if (md == 4) spmv_dots_st_go<TA, T, 2, 4, WIN>(c, d, j, val, rs, pl, s);
        else if (md == 8) spmv_dots_st_go<TA, T, 2, 8, WIN>(c, d, j, val, rs, pl, s);
        else spmv_dots_st_go<TA, T, 2, 16, WIN>(c, d, j, val, rs, pl, s);
        return true;
    }
    return false;
}

template <class TA, class T>
static void spmv_dots_go(Ctx &c, int d, int j, const TA *val, const float *rs, cudaStream_t s) {
    if (c.win && spmv_dots_plan_go<TA, T, true>(c, d, j, val, rs, plan_stage(c, sizeof(TA), c.L[d].m, sizeof(T), sizeof(T)), s))
        return;
    const StagePlan pl = plan_stage(c, sizeof(TA), c.L[d].m, sizeof(T));
    if (!spmv_dots_plan_go<TA, T, false>(c, d, j, val, rs, pl, s)) {
        c.hpart_G[d] = 0;
        launch_pdl(k_spmv_dots<TA, T>, dim3(c.Gs), dim3(kBlock), 0, s, sell_of(c), val, rs, levdev<T>(c, d), j, gred<T>(c, kMaxDots));
    }
}

void launch_spmv_dots(Ctx &c, int d, int j, cudaStream_t s) {
    const float *rs = c.prm.row_scale ? c.rs : nullptr;
    prof_begin(c, PK_SPMV_DOTS, d, s);
    if (c.L[d].v_prec == F3R_F64) {
        spmv_dots_go<double, double>(c, d, j, c.ah64, nullptr, s);
    } else {
        switch (c.L[d].a_prec) {
            case F3R_F32: spmv_dots_go<float, float>(c, d, j, c.a32, nullptr, s); break;
            case F3R_F16: spmv_dots_go<h16, float>(c, d, j, c.a16, rs, s); break;
            default: spmv_dots_go<b16, float>(c, d, j, c.abf, rs, s); break;
        }
    }
    prof_end(c, s);
    c.launches++;
}

template <class T, int MAXD> static void cgs_go(Ctx &c, int d, int j, bool final_pass, bool last, cudaStream_t s) {
    if (final_pass)
        launch_pdl(k_cgs_final<T, MAXD>, dim3(c.Gv), dim3(kVecBlock), 0, s, levdev<T>(c, d), j, c.prm.cgs_passes, last ? 1 : 0,
                                                    want_sigma(c, d), gred<T>(c, kMaxDots));
    else
        launch_pdl(k_cgs_pass<T, MAXD>, dim3(c.Gv), dim3(kVecBlock), 0, s, levdev<T>(c, d), j, gred<T>(c, kMaxDots));
}

template <class T> static void cgs_dispatch(Ctx &c, int d, int j, bool final_pass, bool last, cudaStream_t s) {
    const int md = maxd_bucket(c.L[d].m);
    if (md == 4) cgs_go<T, 4>(c, d, j, final_pass, last, s);
    else if (md == 8) cgs_go<T, 8>(c, d, j, final_pass, last, s);
    else cgs_go<T, 16>(c, d, j, final_pass, last, s);
}

void launch_cgs_pass(Ctx &c, int d, int j, cudaStream_t s) {
    prof_begin(c, PK_CGS_PASS, d, s);
    if (c.L[d].v_prec == F3R_F64) cgs_dispatch<double>(c, d, j, false, false, s);
    else cgs_dispatch<float>(c, d, j, false, false, s);
    prof_end(c, s);
    c.launches++;
}

void launch_cgs_final(Ctx &c, int d, int j, bool last, cudaStream_t s) {
    prof_begin(c, PK_CGS_FINAL, d, s);
    if (c.L[d].v_prec == F3R_F64) cgs_dispatch<double>(c, d, j, true, last, s);
    else cgs_dispatch<float>(c, d, j, true, last, s);
    prof_end(c, s);
    c.launches++;
}

// --------------------------------------------------------------- combine
template <class T, class TP>
static void comb_go(Ctx &c, int d, const OutSlot &o, cudaStream_t s) {
    prof_begin(c, PK_COMBINE, d, s);
    const int md = maxd_bucket(c.L[d].m);
    if (c.L[d].m > kMaxInnerM) {
        launch_pdl(k_combine_long<T, TP>, dim3(c.Gv), dim3(kVecBlock), 0, s, levdev<T>(c, d), (TP *)o.ptr,
                   o.dscale ? c.dsc : nullptr);
    } else {
        auto kern = (md == 4) ? k_combine<T, TP, 4> : (md == 8) ? k_combine<T, TP, 8> : k_combine<T, TP, 16>;
        launch_pdl(kern, dim3(c.Gv), dim3(kVecBlock), 0, s, levdev<T>(c, d), (TP *)o.ptr, nullptr, 0,
                   o.dscale ? c.dsc : nullptr);
    }
    prof_end(c, s);
    c.launches++;
}

void launch_combine(Ctx &c, int d, const OutSlot &o, cudaStream_t s) {
    const bool t64 = c.L[d].v_prec == F3R_F64;
    const bool p64 = o.prec == F3R_F64;
    if (t64 && p64) comb_go<double, double>(c, d, o, s);
    else if (t64) comb_go<double, float>(c, d, o, s);
    else if (p64) comb_go<float, double>(c, d, o, s);
    else comb_go<float, float>(c, d, o, s);
}

// -------------------------------------------------------------------- M
void launch_M(Ctx &c, int d, int j, const void *in, void *out, int check_depth, bool use_j, cudaStream_t s,
              int vround) {
    (void)j;
    const bool t64 = c.L[d].v_prec == F3R_F64;
    unsigned long long *cnt = c.counters;
    const int n = c.n;
    const int *ij = use_j ? c.jdev : nullptr;
    prof_begin(c, PK_M, d, s);
    if (t64) {
        switch (c.prm.m_prec) {
            case F3R_F64: launch_pdl(k_apply_M<double, double>, dim3(c.G), dim3(kBlock), 0, s, (const double *)c.mvec, (const double *)in, ij, c.ld, (double *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
            case F3R_F32: launch_pdl(k_apply_M<double, float>, dim3(c.G), dim3(kBlock), 0, s, (const float *)c.mvec, (const double *)in, ij, c.ld, (double *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
            case F3R_F16: launch_pdl(k_apply_M<double, h16>, dim3(c.G), dim3(kBlock), 0, s, (const h16 *)c.mvec, (const double *)in, ij, c.ld, (double *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
            default: launch_pdl(k_apply_M<double, b16>, dim3(c.G), dim3(kBlock), 0, s, (const b16 *)c.mvec, (const double *)in, ij, c.ld, (double *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
        }
    } else {
        switch (c.prm.m_prec) {
            case F3R_F32: launch_pdl(k_apply_M<float, float>, dim3(c.G), dim3(kBlock), 0, s, (const float *)c.mvec, (const float *)in, ij, c.ld, (float *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
            case F3R_F16: launch_pdl(k_apply_M<float, h16>, dim3(c.G), dim3(kBlock), 0, s, (const h16 *)c.mvec, (const float *)in, ij, c.ld, (float *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
            case F3R_BF16: launch_pdl(k_apply_M<float, b16>, dim3(c.G), dim3(kBlock), 0, s, (const b16 *)c.mvec, (const float *)in, ij, c.ld, (float *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
            default: launch_pdl(k_apply_M<float, double>, dim3(c.G), dim3(kBlock), 0, s, (const double *)c.mvec, (const float *)in, ij, c.ld, (float *)out, n, c.flags, check_depth, (long long *)cnt, vround); break;
        }
    }
    prof_end(c, s);
    c.launches++;
}

// ------------------------------------------------------------ outer level
void launch_outer_residual(Ctx &c, const double *b, const double *x, bool compute_nb, cudaStream_t s) {
    prof_begin(c, PK_OUTER_OTHER, 0, s);
    launch_pdl(k_outer_residual, dim3(c.Gs), dim3(kBlock), 0, s, sell_of(c), c.a64, b, x, levdev<double>(c, 0), gred<double>(c, kMaxDots),
                                              compute_nb ? 1 : 0);
    prof_end(c, s);
    c.launches++;
}

// w = A z (z = the inner nest's output), Z[j] = z, CGS2, Givens, estimate
__global__ void __launch_bounds__(kBlock) k_outer_store_z(LevelDev<double> L, const double *z) {
    pdl_enter();
    const int j = *L.jptr;
    double *dst = L.Z + (size_t)j * L.ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) dst[i] = z[i];
}

// returns true when the fused kernel also normalised V[j+1] (and advanced j)
bool launch_outer_step(Ctx &c, cudaStream_t s) {
    LevelDev<double> L = levdev<double>(c, 0);
    prof_begin(c, PK_OUTER_SPMV, 0, s);
    const StagePlan pw = c.win ? plan_stage(c, sizeof(double), 0, 8, sizeof(double)) : StagePlan();
    const StagePlan pl = plan_stage(c, sizeof(double), 0, 8);
    const Window wn = window_of(c, sizeof(double), c.n);
    if (pw.S == 4) {
        auto kern = k_outer_spmv_st<4, true>;
        const int g = staged_grid(c, kern, pw.smem, ceil_div(c.nslices, kTileSlices));
        launch_pdl(kern, dim3(g), dim3(kStagedThreads), pw.smem, s, sell_of(c), c.a64, L, (const double *)c.zst, StageCfg{pw.stage_bytes, c.err}, wn);
        c.launches--;
    } else if (pw.S == 3) {
        auto kern = k_outer_spmv_st<3, true>;
        const int g = staged_grid(c, kern, pw.smem, ceil_div(c.nslices, kTileSlices));
        launch_pdl(kern, dim3(g), dim3(kStagedThreads), pw.smem, s, sell_of(c), c.a64, L, (const double *)c.zst, StageCfg{pw.stage_bytes, c.err}, wn);
        c.launches--;
    } else if (pw.S == 2) {
        auto kern = k_outer_spmv_st<2, true>;
        const int g = staged_grid(c, kern, pw.smem, ceil_div(c.nslices, kTileSlices));
        launch_pdl(kern, dim3(g), dim3(kStagedThreads), pw.smem, s, sell_of(c), c.a64, L, (const double *)c.zst, StageCfg{pw.stage_bytes, c.err}, wn);
        c.launches--;
    } else if (pl.S == 3) {
        auto kern = k_outer_spmv_st<3>;
        const int g = staged_grid(c, kern, pl.smem, ceil_div(c.nslices, kTileSlices));
        launch_pdl(kern, dim3(g), dim3(kStagedThreads), pl.smem, s, sell_of(c), c.a64, L, (const double *)c.zst, StageCfg{pl.stage_bytes, c.err}, Window());
        c.launches--;
    } else if (pl.S == 2) {
        auto kern = k_outer_spmv_st<2>;
        const int g = staged_grid(c, kern, pl.smem, ceil_div(c.nslices, kTileSlices));
        launch_pdl(kern, dim3(g), dim3(kStagedThreads), pl.smem, s, sell_of(c), c.a64, L, (const double *)c.zst, StageCfg{pl.stage_bytes, c.err}, Window());
        c.launches--;
    } else {
        launch_pdl(k_outer_store_z, dim3(c.G), dim3(kBlock), 0, s, L, (const double *)c.zst);
        launch_pdl(k_outer_spmv, dim3(c.Gs), dim3(kBlock), 0, s, sell_of(c), c.a64, L);
    }
    prof_end(c, s);
    if (launch_outer_cgs_fused(c, s)) return true;
    double *part = (double *)c.partials;
    prof_begin(c, PK_OUTER_CGS, 0, s);
    launch_pdl(k_outer_cgs<0>, dim3(c.G1), dim3(512), 0, s, L, c.prm.cgs_passes, part, c.ticket);
    c.launches += 3;
    if (c.prm.cgs_passes == 2) {
        launch_pdl(k_outer_cgs<1>, dim3(c.G1), dim3(512), 0, s, L, c.prm.cgs_passes, part, c.ticket);
        c.launches++;
    }
    launch_pdl(k_outer_cgs<2>, dim3(c.G1), dim3(512), 0, s, L, c.prm.cgs_passes, part, c.ticket);
    prof_end(c, s);
    c.launches++;
    return false;
}

void launch_outer_finish(Ctx &c, double *x, cudaStream_t s) {
    LevelDev<double> L = levdev<double>(c, 0);
    prof_begin(c, PK_OUTER_OTHER, 0, s);
    launch_pdl(k_outer_solve_y, dim3(1), dim3(32), 0, s, L);
    launch_pdl(k_outer_update_x, dim3(c.G), dim3(kBlock), 0, s, L, x);
    prof_end(c, s);
    c.launches += 2;
}

__global__ void k_advance(long long *p, long long inc) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) *p += inc;
}

void launch_advance(Ctx &c, long long inc, cudaStream_t s) {
    prof_begin(c, PK_OUTER_OTHER, 0, s);
    launch_pdl(k_advance, dim3(1), dim3(32), 0, s, c.c_ntr_base, inc);
    prof_end(c, s);
    c.launches++;
}

// ------------------------------------------------------- stand-alone SpMV
template <class TA, class TX, class TY>
__global__ void __launch_bounds__(kBlock) k_spmv(Sell S, const TA *__restrict__ val, const float *__restrict__ rs,
                                                 const TX *__restrict__ x, TY *y) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        TY acc = sell_row<TY>(S, val, s, lane, [&](int c) { return to_c<TY>(__ldg(x + c)); });
        const int i = s * kSlice + lane;
        if (rs) acc = mul_rn(acc, (TY)__ldg(rs + i));
        if (i < S.n) y[i] = acc;
    }
}

template <class TA, class TX, class TY>
static void spmv_go(Ctx &c, const TA *val, const float *rs, const TX *x, TY *y, cudaStream_t s) {
    // the window's bulk copies read x from 16-byte aligned addresses (a caller's
    // x at another offset is gathered from global memory instead)
    const bool xal = ((uintptr_t)x % 16) == 0;
    const StagePlan pw = (c.win && xal) ? plan_stage(c, sizeof(TA), 0, 4, sizeof(TX)) : StagePlan();
    const StagePlan pl = plan_stage(c, sizeof(TA), 0, 4);
    const StageCfg cfg{pl.stage_bytes, c.err};
    const StageCfg cfw{pw.stage_bytes, c.err};
    const int work = ceil_div(c.nslices, kTileSlices);
    if (pw.S == 4) {
        auto kern = k_spmv_st<TA, TX, TY, 4, true>;
        launch_pdl(kern, dim3(staged_grid(c, kern, pw.smem, work)), dim3(kStagedThreads), pw.smem, s, sell_of(c), val, rs, x, y,
                   cfw, window_of(c, sizeof(TX), c.n));
    } else if (pw.S == 3) {
        auto kern = k_spmv_st<TA, TX, TY, 3, true>;
        launch_pdl(kern, dim3(staged_grid(c, kern, pw.smem, work)), dim3(kStagedThreads), pw.smem, s, sell_of(c), val, rs, x, y,
                   cfw, window_of(c, sizeof(TX), c.n));
    } else if (pw.S == 2) {
        auto kern = k_spmv_st<TA, TX, TY, 2, true>;
        launch_pdl(kern, dim3(staged_grid(c, kern, pw.smem, work)), dim3(kStagedThreads), pw.smem, s, sell_of(c), val, rs, x, y,
                   cfw, window_of(c, sizeof(TX), c.n));
    } else if (pl.S == 3) {
        auto kern = k_spmv_st<TA, TX, TY, 3>;
        launch_pdl(kern, dim3(staged_grid(c, kern, pl.smem, work)), dim3(kStagedThreads), pl.smem, s, sell_of(c), val, rs,
                                                                                                x, y, cfg, Window());
    } else if (pl.S == 2) {
        auto kern = k_spmv_st<TA, TX, TY, 2>;
        launch_pdl(kern, dim3(staged_grid(c, kern, pl.smem, work)), dim3(kStagedThreads), pl.smem, s, sell_of(c), val, rs,
                                                                                                x, y, cfg, Window());
    } else {
        launch_pdl(k_spmv<TA, TX, TY>, dim3(c.Gs), dim3(kBlock), 0, s, sell_of(c), val, rs, x, y);
    }
}

f3r_status launch_spmv(Ctx &c, int p, int vp, const void *x, void *y, cudaStream_t s) {
    const float *rs = c.prm.row_scale ? c.rs : nullptr;
    f3r_status st = F3R_OK;
    prof_begin(c, PK_SPMV, p, s);
    switch (p) {
        case F3R_F64:
            if (vp != F3R_F64) st = F3R_ERR_ARG;
            else spmv_go<double, double, double>(c, c.a64, nullptr, (const double *)x, (double *)y, s);
            break;
        case F3R_F32:
            if (!c.a32 || vp != F3R_F32) st = F3R_ERR_ARG;
            else spmv_go<float, float, float>(c, c.a32, nullptr, (const float *)x, (float *)y, s);
            break;
        case F3R_F16:
            if (!c.a16) st = F3R_ERR_ARG;
            else if (vp == F3R_F32) spmv_go<h16, float, float>(c, c.a16, rs, (const float *)x, (float *)y, s);
            else if (vp == F3R_F16) spmv_go<h16, h16, float>(c, c.a16, rs, (const h16 *)x, (float *)y, s);
            else st = F3R_ERR_ARG;
            break;
        case F3R_BF16:
            if (!c.abf) st = F3R_ERR_ARG;
            else if (vp == F3R_F32) spmv_go<b16, float, float>(c, c.abf, rs, (const float *)x, (float *)y, s);
            else if (vp == F3R_BF16) spmv_go<b16, b16, float>(c, c.abf, rs, (const b16 *)x, (float *)y, s);
            else st = F3R_ERR_ARG;
            break;
        default:
            st = F3R_ERR_ARG;
    }
    prof_end(c, s);
    if (st == F3R_OK) c.launches++;
    return st;
}

// --------------------------------------------------- long inner levels
// One iteration's w = A_l Z[j] and CGS2 + Givens of a level with m > kMaxInnerM.
template <class T> static void long_cgs_go(Ctx &c, int d, int j, bool last, cudaStream_t s) {
    const LevelDev<T> L = levdev<T>(c, d);
    T *part = (T *)c.partials;
    const int ws = want_sigma(c, d), passes = c.prm.cgs_passes, li = last ? 1 : 0;
    // two blocks per SM at most: [vector][block] partials fit the scratch (kMaxLongM + 1 rows)
    const int g = std::max(1, std::min(ceil_div(c.n / (16 / (int)sizeof(T)), kLongBlock), 2 * c.nsm));
    launch_pdl(k_long_cgs<T, 0>, dim3(g), dim3(kLongBlock), 0, s, L, j, passes, li, ws, part, c.ticket, gred<T>(c, kMaxDots));
    if (passes == 2) {
        launch_pdl(k_long_cgs<T, 1>, dim3(g), dim3(kLongBlock), 0, s, L, j, passes, li, ws, part, c.ticket, gred<T>(c, kMaxDots));
        c.launches++;
    }
    launch_pdl(k_long_cgs<T, 2>, dim3(g), dim3(kLongBlock), 0, s, L, j, passes, li, ws, part, c.ticket, gred<T>(c, kMaxDots));
    c.launches += 2;
}

void launch_long_step(Ctx &c, int d, int j, bool last, cudaStream_t s) {
    const LevelHost &H = c.L[d];
    const float *rs = c.prm.row_scale ? c.rs : nullptr;
    const char *z = (const char *)H.Z + (size_t)j * c.ld * level_vec_bytes(c, d);
    prof_begin(c, PK_SPMV_DOTS, d, s);
    if (H.v_prec == F3R_F64) {
        spmv_go<double, double, double>(c, c.ah64, nullptr, (const double *)z, (double *)H.w, s);
    } else {
        switch (H.a_prec) {
            case F3R_F32: spmv_go<float, float, float>(c, c.a32, nullptr, (const float *)z, (float *)H.w, s); break;
            case F3R_F16: spmv_go<h16, float, float>(c, c.a16, rs, (const float *)z, (float *)H.w, s); break;
            default: spmv_go<b16, float, float>(c, c.abf, rs, (const float *)z, (float *)H.w, s); break;
        }
    }
    prof_end(c, s);
    c.launches++;
    prof_begin(c, PK_CGS_FINAL, d, s);
    if (H.v_prec == F3R_F64) long_cgs_go<double>(c, d, j, last, s);
    else long_cgs_go<float>(c, d, j, last, s);
    prof_end(c, s);
}

}  // namespace f3r
