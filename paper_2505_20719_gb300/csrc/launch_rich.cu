// Launchers of the Richardson level (Algorithm 1), dispatching on the
// storage of A and of the Richardson vectors.
#include <algorithm>

#include "ctx.h"
#include "rich.cuh"
#include "staged.cuh"

namespace f3r {

template <class TC> static RichDev<TC> richdev(Ctx &c) {
    return RichDev<TC>{(TC *)c.omega, (TC *)c.wcur, c.counters, c.c_ntr_base};
}

template <class K> static int rich_grid(Ctx &c, K kern, int smem) {
    ensure_dyn_smem((const void *)kern, smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kStagedThreads, smem);
    nb = std::max(1, std::min(nb, 8));
    return std::max(1, std::min(c.nsm * nb, ceil_div(c.nslices, kTileSlices)));
}

template <class TA, class VS, class TC, class TP>
static void rich_go(Ctx &c, const TA *val, bool update, int pos, TP *out, const TP *par_misc, cudaStream_t s) {
    const Sell S = sell_of(c);
    const float *rs = (c.prm.row_scale && IsHalfWidth<TA>::value) ? c.rs : nullptr;
    const VS *v = (const VS *)c.rin;
    const VS *mv = (const VS *)c.mvec;
    const int m4 = c.prm.rich_m, n = c.n;
    const int cd = c.prm.nlevels - 1;
    RichDev<TC> R = richdev<TC>(c);
    VS *zb[2] = {(VS *)c.rz[0], (VS *)c.rz[1]};
    if (!update) {
        if (m4 == 2) {
            prof_begin(c, PK_RICH2, 0, s);
            const StagePlan pw = (c.win && c.m_unit) ? plan_stage(c, sizeof(TA), 0, 4, sizeof(VS)) : StagePlan();
            const StagePlan pl = plan_stage(c, sizeof(TA), 0, 4);
            const StageCfg cfg{pl.stage_bytes, c.err};
            const StageCfg cfw{pw.stage_bytes, c.err};
            const Window wn = window_of(c, sizeof(VS), n);
            if (pw.S == 4) {
                auto kern = k_rich2_st<TA, VS, TC, TP, 4, true, true>;
                launch_pdl(kern, dim3(rich_grid(c, kern, pw.smem)), dim3(kStagedThreads), pw.smem, s, S, val, rs, v, mv, out,
                           par_misc, R, c.flags, cd, n, cfw, wn);
            } else if (pw.S == 3) {
                auto kern = k_rich2_st<TA, VS, TC, TP, 3, true, true>;
                launch_pdl(kern, dim3(rich_grid(c, kern, pw.smem)), dim3(kStagedThreads), pw.smem, s, S, val, rs, v, mv, out,
                           par_misc, R, c.flags, cd, n, cfw, wn);
            } else if (pw.S == 2) {
                auto kern = k_rich2_st<TA, VS, TC, TP, 2, true, true>;
                launch_pdl(kern, dim3(rich_grid(c, kern, pw.smem)), dim3(kStagedThreads), pw.smem, s, S, val, rs, v, mv, out,
                           par_misc, R, c.flags, cd, n, cfw, wn);
            } else if (pl.S == 3 && c.m_unit) {
                auto kern = k_rich2_st<TA, VS, TC, TP, 3, true>;
                launch_pdl(kern, dim3(rich_grid(c, kern, pl.smem)), dim3(kStagedThreads), pl.smem, s, S, val, rs, v, mv, out, par_misc, R, c.flags,
                                                                          cd, n, cfg, Window());
            } else if (pl.S == 3) {
                auto kern = k_rich2_st<TA, VS, TC, TP, 3>;
                launch_pdl(kern, dim3(rich_grid(c, kern, pl.smem)), dim3(kStagedThreads), pl.smem, s, S, val, rs, v, mv, out, par_misc, R, c.flags,
                                                                          cd, n, cfg, Window());
            } else if (pl.S == 2) {
                auto kern = k_rich2_st<TA, VS, TC, TP, 2>;
                launch_pdl(kern, dim3(rich_grid(c, kern, pl.smem)), dim3(kStagedThreads), pl.smem, s, S, val, rs, v, mv, out, par_misc, R, c.flags,
                                                                          cd, n, cfg, Window());
            } else {
                launch_pdl(k_rich2<TA, VS, TC, TP>, dim3(c.Gs), dim3(kBlock), 0, s, S, val, rs, v, mv, out, par_misc, R, c.flags, cd, n);
            }
            prof_end(c, s);
            c.launches++;
        } else {
            for (int k = 0; k < m4; ++k) {
                const bool last = (k == m4 - 1);
                const VS *zp = (k > 0) ? zb[(k - 1) & 1] : nullptr;
                prof_begin(c, PK_RICH_STEP, 0, s);
                launch_pdl(k_rich_step<TA, VS, TC, TP>, dim3(c.Gs), dim3(kBlock), 0, s, S, val, rs, v, mv, zp, zb[k & 1], out, par_misc,
                                                                    R, k, last ? 1 : 0, c.flags, cd, n);
                prof_end(c, s);
                c.launches++;
            }
        }
        return;
    }
    // update call: every step computes w'_k (Algorithm 1, update branch)
    VS *r = (VS *)c.rr;
    GridRed<TC> gr{(TC *)c.partials, c.ticket, kMaxDots};
    for (int k = 0; k < m4; ++k) {
        const bool last = (k == m4 - 1);
        const VS *zp = (k > 0) ? zb[(k - 1) & 1] : nullptr;
        const VS *rk = v;  // r_0 = v without an SpMV
        prof_begin(c, PK_RICH_UPD, 0, s);
        if (k > 0) {
            launch_pdl(k_rich_upd_r<TA, VS, TC>, dim3(c.Gs), dim3(kBlock), 0, s, S, val, rs, v, zp, r, c.flags, cd, n);
            rk = r;
            c.launches++;
        }
        launch_pdl(k_rich_upd_w<TA, VS, TC>, dim3(c.Gs), dim3(kBlock), 0, s, S, val, rs, rk, mv, R, k, pos, c.prm.c, gr, c.flags, cd, n);
        launch_pdl(k_rich_upd_z<VS, TC, TP>, dim3(c.G), dim3(kBlock), 0, s, rk, mv, zp, zb[k & 1], out, par_misc, R, last ? 1 : 0,
                                                       c.flags, cd, n);
        prof_end(c, s);
        c.launches += 2;
    }
}

void launch_rich_call(Ctx &c, bool update, int pos, void *out, const void *par_misc, cudaStream_t s) {
    const int a = c.prm.rich_a_prec, v = c.prm.rich_v_prec;
    if (c.prm.precond == F3R_PC_AINV) {
        prof_begin(c, PK_RICH_STEP, 2, s);
        ainv_rich_call(c, update, pos, out, par_misc, s);
        prof_end(c, s);
        return;
    }
    if (c.prm.precond == F3R_PC_LEARNED && c.learned) {
        prof_begin(c, PK_RICH_STEP, 1, s);
        learned_rich_call(c, update, pos, out, par_misc, s);
        prof_end(c, s);
        return;
    }
    if (v == F3R_F16 && a == F3R_F16)
        rich_go<h16, h16, float, float>(c, c.a16, update, pos, (float *)out, (const float *)par_misc, s);
    else if (v == F3R_BF16 && a == F3R_BF16)
        rich_go<b16, b16, float, float>(c, c.abf, update, pos, (float *)out, (const float *)par_misc, s);
    else if (v == F3R_F32 && a == F3R_F32)
        rich_go<float, float, float, float>(c, c.a32, update, pos, (float *)out, (const float *)par_misc, s);
    else if (v == F3R_F64 && a == F3R_F64)
        rich_go<double, double, double, double>(c, c.ah64, update, pos, (double *)out, (const double *)par_misc, s);
}

// Stand-alone call: sigma from max|x|, then the cast into the Richardson input.
void launch_rich_prep(Ctx &c, const void *x, cudaStream_t s) {
    const bool p64 = c.L[c.prm.nlevels - 1].v_prec == F3R_F64;
    const int ws = (c.prm.scale_cast && (c.prm.rich_v_prec == F3R_F16 || c.prm.rich_v_prec == F3R_BF16)) ? 1 : 0;
    if (p64) {
        GridRed<double> gr{(double *)c.partials, c.ticket, kMaxDots};
        launch_pdl(k_amax_sigma<double>, dim3(c.G), dim3(kBlock), 0, s, (const double *)x, c.n, (double *)c.apply_misc, ws, gr);
        launch_pdl(k_cast_scaled<double, double>, dim3(c.G), dim3(kBlock), 0, s, (const double *)x, (double *)c.rin, c.n,
                                                              (const double *)c.apply_misc);
    } else {
        GridRed<float> gr{(float *)c.partials, c.ticket, kMaxDots};
        launch_pdl(k_amax_sigma<float>, dim3(c.G), dim3(kBlock), 0, s, (const float *)x, c.n, (float *)c.apply_misc, ws, gr);
        switch (c.prm.rich_v_prec) {
            case F3R_F16:
                launch_pdl(k_cast_scaled<float, h16>, dim3(c.G), dim3(kBlock), 0, s, (const float *)x, (h16 *)c.rin, c.n,
                                                                 (const float *)c.apply_misc);
                break;
            case F3R_BF16:
                launch_pdl(k_cast_scaled<float, b16>, dim3(c.G), dim3(kBlock), 0, s, (const float *)x, (b16 *)c.rin, c.n,
                                                                 (const float *)c.apply_misc);
                break;
            default:
                launch_pdl(k_cast_scaled<float, float>, dim3(c.G), dim3(kBlock), 0, s, (const float *)x, (float *)c.rin, c.n,
                                                                   (const float *)c.apply_misc);
                break;
        }
    }
    c.launches += 2;
}

}  // namespace f3r
