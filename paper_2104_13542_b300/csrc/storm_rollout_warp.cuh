// storm_rollout_warp.cuh -- sample_controls + generate_rollouts with one lane
// per (particle, step) item.
//
// A particle's horizon lies along one segment of Lp = 8, 16 or 32 lanes of a
// warp (Lp >= H, or Lp = 32 with ceil(H / 32) items per lane), so each phase
// runs on all the particle's items at once and the only synchronisation is the
// warp's own.  Per-item results are bitwise those of the CTA-wide mapping in
// k_rollout: the same noise, the same sequential integration (one lane per
// (particle, joint)), the same FK / Jacobian / cost expressions, exact sphere
// tests with the same formulas, and the same sequential discounted sum.  What
// changes is the work schedule: no CTA barriers, Jacobian and bounding-sphere
// centres in registers, world obstacles culled once per warp against the
// axis-aligned box enclosing every link bound of the warp's items, and self
// collision culled by link capsules (segment + radius) after the spheres.
//
// The pair and quad variants (kW = 2 or 4 warps per particle group) split
// each item's work across warps.  Warp A draws the controls and integrates
// them; then every warp of the group runs FK into its own copy of the link
// frames.  Pair: A takes the pose, joint and end-effector terms and world
// collision, B the manipulability term and self collision, and A, once its
// own terms are done, joins in: B publishes each item's mask of overlapping frame pairs in
// shared memory, and the pairs are claimed one at a time from a per-item
// counter, B from the first pair, A from the last, so that every pair is
// tested exactly once and the two warps finish together however the work
// falls (the arm folded onto itself makes self collision several times the
// rest of the item's work).  Quad: A the pose, joint and
// end-effector terms, B world collision and manipulability, C and D alternate
// halves of each lane's overlapping self-collision frame pairs.  The warps
// meet at one named barrier per step slot, where A gathers the depths (a max
// over the same tests, in any order) and adds the terms in the single-warp
// order; the critical path is the longest branch, not their sum.
#pragma once

// Per-warp shared-memory plan (float offsets).
struct WarpPlan {
    int Lp, PW, SL;  // lanes per particle, particles per warp, items per lane
    int frame;       // kW x F x 12 x 32: link frames, row-major [R | p] rows, lane-minor, one copy per warp
    int fstride;     // one warp's frame copy
    int eps;         // PW x S x d noise
    int u, th, thd;  // PW x H x d controls and joint states
    int c;           // PW x H running costs
    int ba;          // PW x H x 2 ball in-plane gravity
    int hand;        // 4 x PW x H handed to warp A: self depths (C, D), world depth, manipulability cost
    int lpb;         // kLinkPairs + 1 ints: the frame pairs' block ranges (Problem::lp_begin)
    int claim;       // 3 x SL x 32 ints (pair mapping), per item: B's mask of the overlapping frame pairs
                     // (bit 31: published), the pairs B has started (from the first), A has started
                     // (from the last)
    int io;          // mu (H x d) | sigma (d) | state (3 x d) | goal (7) | dt (H) | gamma^h (H) |
                     // B-spline basis (H x nk), staged per warp
    int floats;      // size of one warp's (pair's) region
};

__host__ __device__ inline WarpPlan warp_plan(const Problem& pb, int kw)
{
    WarpPlan w;
    w.Lp = pb.H > 16 ? 32 : (pb.H > 8 ? 16 : 8);
    w.PW = 32 / w.Lp;
    w.SL = (pb.H + w.Lp - 1) / w.Lp;
    const int F = pb.d + 1;
    int off = 0;
    auto take = [&](int n) {
        const int o = off;
        off += (n + 3) & ~3;
        return o;
    };
    w.fstride = F * 12 * 32;
    w.frame = take(kw * w.fstride);
    w.eps = take(w.PW * pb.S * pb.d);
    w.u = take(w.PW * pb.H * pb.d);
    w.th = take(w.PW * pb.H * pb.d);
    w.thd = take(w.PW * pb.H * pb.d);
    w.c = take(w.PW * pb.H);
    w.ba = take(w.PW * pb.H * 2);
    w.hand = take(4 * w.PW * pb.H);
    w.lpb = take(kLinkPairs + 1);
    w.claim = take(3 * w.SL * 32);
    w.io = take(pb.H * pb.d + 4 * pb.d + 7 + 2 * pb.H + pb.H * pb.nk);
    w.floats = off;
    return w;
}

constexpr int kWarpMaxWarps = 8;  // largest CTA of the warp mapping (warps)

// Asynchronous 4-byte copy global -> shared (completed by cp.async.wait_all).
__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}

// Exact depth of the spheres [s0, s1) of one frame against box b (centre,
// half extents) -- the per-sphere formula of k_rollout.
__device__ __forceinline__ float box_depth(const float* __restrict__ fr, int lane, const float4* __restrict__ sph,
                                           int s0, int s1, const float* __restrict__ box, float depth)
{
    const float r0x = fr[0 * 32 + lane], r0y = fr[1 * 32 + lane], r0z = fr[2 * 32 + lane], r0w = fr[3 * 32 + lane];
    const float r1x = fr[4 * 32 + lane], r1y = fr[5 * 32 + lane], r1z = fr[6 * 32 + lane], r1w = fr[7 * 32 + lane];
    const float r2x = fr[8 * 32 + lane], r2y = fr[9 * 32 + lane], r2z = fr[10 * 32 + lane], r2w = fr[11 * 32 + lane];
    const float lox = box[0] - box[3], loy = box[1] - box[4], loz = box[2] - box[5];
    const float hix = box[0] + box[3], hiy = box[1] + box[4], hiz = box[2] + box[5];
    for (int s = s0; s < s1; ++s) {
        const float4 q = sph[s];
        const float cx = fmaf(r0x, q.x, fmaf(r0y, q.y, fmaf(r0z, q.z, r0w)));
        const float cy = fmaf(r1x, q.x, fmaf(r1y, q.y, fmaf(r1z, q.z, r1w)));
        const float cz = fmaf(r2x, q.x, fmaf(r2y, q.y, fmaf(r2z, q.z, r2w)));
        const float fx = cx - fminf(fmaxf(cx, lox), hix);
        const float fy = cy - fminf(fmaxf(cy, loy), hiy);
        const float fz = cz - fminf(fmaxf(cz, loz), hiz);
        if (fmaf(fx, fx, fmaf(fy, fy, fz * fz)) < q.w * q.w) {
            const float qx = fabsf(cx - box[0]) - box[3];
            const float qy = fabsf(cy - box[1]) - box[4];
            const float qz = fabsf(cz - box[2]) - box[5];
            const float ox = fmaxf(qx, 0.f), oy = fmaxf(qy, 0.f), oz = fmaxf(qz, 0.f);
            const float sd = sqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) + fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f) - q.w;
            depth = fmaxf(depth, -sd);
        }
    }
    return depth;
}

// Exact depth of the spheres [s0, s1) of one frame against obstacle sphere w.
__device__ __forceinline__ float ball_depth(const float* __restrict__ fr, int lane, const float4* __restrict__ sph,
                                            int s0, int s1, float4 w, float depth)
{
    const float r0x = fr[0 * 32 + lane], r0y = fr[1 * 32 + lane], r0z = fr[2 * 32 + lane], r0w = fr[3 * 32 + lane];
    const float r1x = fr[4 * 32 + lane], r1y = fr[5 * 32 + lane], r1z = fr[6 * 32 + lane], r1w = fr[7 * 32 + lane];
    const float r2x = fr[8 * 32 + lane], r2y = fr[9 * 32 + lane], r2z = fr[10 * 32 + lane], r2w = fr[11 * 32 + lane];
    for (int s = s0; s < s1; ++s) {
        const float4 q = sph[s];
        const float cx = fmaf(r0x, q.x, fmaf(r0y, q.y, fmaf(r0z, q.z, r0w)));
        const float cy = fmaf(r1x, q.x, fmaf(r1y, q.y, fmaf(r1z, q.z, r1w)));
        const float cz = fmaf(r2x, q.x, fmaf(r2y, q.y, fmaf(r2z, q.z, r2w)));
        const float gx = cx - w.x, gy = cy - w.y, gz = cz - w.z;
        const float dist2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
        const float rs = q.w + w.w;
        if (dist2 < rs * rs) depth = fmaxf(depth, rs - sqrtf(dist2));
    }
    return depth;
}

// World collision without the broad phase: every sphere of every frame against
// every obstacle (the same tests in the same order as the inline form).  Out of
// line, so that this cold path does not sit in the hot instruction stream.
__device__ __noinline__ float world_brute_force(const float* __restrict__ s_fr, int lane,
                                                const int* __restrict__ link_first, const float4* __restrict__ sph,
                                                int F, const float* __restrict__ boxes, int B,
                                                const float4* __restrict__ wsph, int O, float dworld)
{
    for (int f = 0; f < F; ++f) {
        const int s0 = link_first[f], s1 = link_first[f + 1];
        if (s0 >= s1) continue;
        for (int b = 0; b < B; ++b) dworld = box_depth(s_fr + f * 12 * 32, lane, sph, s0, s1, boxes + b * 6, dworld);
        for (int k = 0; k < O; ++k) dworld = ball_depth(s_fr + f * 12 * 32, lane, sph, s0, s1, wsph[k], dworld);
    }
    return dworld;
}

// The ball along one particle's horizon (initial state from the current pose, then
// the scan), out of line: only ball-balancing problems take it.
__device__ __noinline__ void ball_tail(const float* dhx, int d, const float* state, const float* ball, int H,
                                       float w_ball, float tray_x, float tray_y, const float* a, const float* dt,
                                       float* c, float* term)
{
    const float4 s0 = ball_initial(dhx, d, state, ball);
    ball_scan(H, w_ball, tray_x, tray_y, s0, a, dt, c, term, STORM_NTERMS);
}

// Centre of sphere q in frame fr (the k_rollout expression).
__device__ __forceinline__ float3 frame_point(const float* __restrict__ fr, int lane, float4 q)
{
    return make_float3(fmaf(fr[0 * 32 + lane], q.x, fmaf(fr[1 * 32 + lane], q.y, fmaf(fr[2 * 32 + lane], q.z, fr[3 * 32 + lane]))),
                       fmaf(fr[4 * 32 + lane], q.x, fmaf(fr[5 * 32 + lane], q.y, fmaf(fr[6 * 32 + lane], q.z, fr[7 * 32 + lane]))),
                       fmaf(fr[8 * 32 + lane], q.x, fmaf(fr[9 * 32 + lane], q.y, fmaf(fr[10 * 32 + lane], q.z, fr[11 * 32 + lane]))));
}

// The warps of group `unit` meet (named barrier 1 + unit, `threads` threads).
__device__ __forceinline__ void unit_sync(int unit, int threads)
{
    asm volatile("barrier.sync %0, %1;" ::"r"(unit + 1), "r"(threads) : "memory");
}

// The rollout of particle group `wg` (particles wg*PW ..) of problem pb by
// this warp (or the kW warps of group `unit`), in the group's shared-memory
// region ws.  kFull: the end-effector limit terms, the ball, the comb / mixed
// filters, the Halton sampler, the Frobenius rotation cost, the learned
// self-collision term and the per-item outputs of the single-stage calls are
// compiled in; a problem without them (Philox noise, the default filter, the
// quaternion rotation cost, exact self collision) runs the lean instantiation,
// without that code in its instruction stream.
// kPhase: 0 the whole rollout; 1 up to the joint states (noise, controls,
// Eq. 7); 2 the rest, on the joint states phase 1 left in ws.  lane_pred (phase
// 2 or kFull; nullable): the learned self-collision network's output for this
// lane's items, item slot s at lane_pred[s * kMlpRows] (pb.self_mode says how
// it is used).
template <int kW, bool kFull, int kPhase = 0>
__device__ __forceinline__ void rollout_warp_body(const Problem& pb, const RolloutOut& out,
                                                  const float* __restrict__ state, const float* __restrict__ goal,
                                                  uint32_t step, int iter, int wg, int unit, float* ws,
                                                  const float* lane_pred = nullptr)
{
    static_assert(kW == 1 || kW == 2 || kW == 4, "one, two or four warps per particle group");
    const WarpPlan W = warp_plan(pb, kW);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int role = kW == 1 ? 0 : warp % kW;
    const bool do_costs = role == 0;  // A: controls, integration, the cost terms
    const bool do_world = kW == 1 || (kW == 2 ? role == 0 : role == 1);
    const bool do_manipw = kW == 1 || role == 1;  // pair and quad: B (A's chain is the longer)
    // self collision: the single warp; both warps of a pair (B takes each item's
    // overlapping frame pairs from the first, A, once its own terms are done,
    // from the last, one claim at a time); the quad's C and D (alternate pairs)
    const bool do_selfc = kW <= 2 || role >= 2;
    const int self_half = kW == 4 ? role - 2 : -1;  // quad: which alternate hits; -1: all of them
    const int nw0 = wg * W.PW;  // first particle of this unit
    if (nw0 >= pb.N) return;    // uniform over the unit (all its warps)
    if (kPhase != 2 && kW == 2 && role == 1)   // (ordered before any claim by the unit barrier after the prefix)
        for (int i = lane; i < 3 * W.SL * 32; i += 32) reinterpret_cast<int*>(ws + W.claim)[i] = 0;
    if (kPhase != 2 && (kW == 1 || role == 1)) {  // the block ranges, for reads at an item's own frame pairs
        static_assert(kLinkPairs < 32, "one lane per frame pair");
        int v = 0;
#pragma unroll
        for (int u = 0; u <= kLinkPairs; ++u)
            if (u == lane) v = pb.lp_begin[u];
        if (lane <= kLinkPairs) reinterpret_cast<int*>(ws + W.lpb)[lane] = v;
    }
    float* s_fr = ws + W.frame + role * W.fstride;  // this warp's own frames
    float* s_eps = ws + W.eps;
    float* s_u = ws + W.u;
    float* s_th = ws + W.th;
    float* s_thd = ws + W.thd;
    float* s_c = ws + W.c;
    const int d = pb.d, H = pb.H, S = pb.S, F = d + 1, Lp = W.Lp, HD = H * d;
    const int seg = lane / Lp, hl = lane - seg * Lp;
    const int np_w = min(W.PW, pb.N - nw0);
    const int n = nw0 + seg;
    const bool pvalid = seg < np_w;
    trace_stamp(pb.trace, 0);
    // mu, sigma, the state and the goal: read by every lane, so staged with one
    // coalesced pass per warp (the whole grid reads these same few lines)
    float* s_mu = ws + W.io;
    float* s_sig = s_mu + H * d;
    float* s_st = s_sig + d;
    float* s_goal = s_st + 3 * d;
    float* s_dt = s_goal + 7;  // the time steps and discount powers, read in dependent chains
    float* s_gp = s_dt + H;
    float* s_basis = s_gp + H;  // H x nk
    const int mu_off = (pb.shift_view && step > 0) ? d : 0;  // the shifted mean at a step's start
    auto stage_inputs = [&]() {
        for (int i = lane; i < H * d; i += 32) s_mu[i] = i + mu_off < H * d ? __ldcg(pb.mu + i + mu_off) : 0.f;
        if (lane < d) s_sig[lane] = __ldcg(pb.sigma + lane);
        if (lane < 3 * d) s_st[lane] = state[lane];
        if (lane < 7) s_goal[lane] = goal[lane];
        for (int i = lane; i < H; i += 32) {
            s_dt[i] = pb.dt[i];
            s_gp[i] = pb.gpow[i];
        }
        for (int i = lane; i < H * pb.nk; i += 32) s_basis[i] = pb.basis[i];
    };
    auto stage_inputs_async = [&]() {  // the same copies, in flight while the noise is drawn
        for (int i = lane; i < H * d; i += 32) {
            if (i + mu_off < H * d)
                cp_async4(s_mu + i, pb.mu + i + mu_off);
            else
                s_mu[i] = 0.f;
        }
        if (lane < d) cp_async4(s_sig + lane, pb.sigma + lane);
        if (lane < 3 * d) cp_async4(s_st + lane, state + lane);
        if (lane < 7) cp_async4(s_goal + lane, goal + lane);
        for (int i = lane; i < H; i += 32) {
            cp_async4(s_dt + i, pb.dt + i);
            cp_async4(s_gp + i, pb.gpow + i);
        }
        for (int i = lane; i < H * pb.nk; i += 32) cp_async4(s_basis + i, pb.basis + i);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (kPhase != 2 && do_costs) {
    // launched ordinarily, the inputs are final: their loads overlap the noise
    // (issued first: the controls wait on them)
    if (!pb.dep_launch) stage_inputs_async();
    {
        // The grid is a single wave, so every warp meets this SM's L1 cold: pull
        // the read-only tables into it now, while the noise is drawn, rather
        // than one dependent miss at a time later.
        const char* tb = reinterpret_cast<const char*>(pb.tables);
        for (int o = lane * 128; o < pb.table_bytes; o += 32 * 128)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(tb + o));
    }

    // ---- noise eps[n][s][j] of the warp's particles
    const int per = S * d;
    if (!kFull || pb.sampler == STORM_SAMPLER_PHILOX) {
        const uint32_t e0 = static_cast<uint32_t>(nw0) * per;
        const uint32_t e1 = static_cast<uint32_t>(nw0 + np_w) * per;
        const uint32_t b0 = e0 >> 2, b1 = (e1 + 3) >> 2;
        const uint32_t c2 = (pb.instance << 8) | static_cast<uint32_t>(iter);
        for (uint32_t b = b0 + lane; b < b1; b += 32) {
            const uint4 x = philox4x32_10(make_uint4(b, step, c2, 0u), pb.seed_lo, pb.seed_hi);
            const float2 z01 = gauss_pair(x.x, x.y);
            const float2 z23 = gauss_pair(x.z, x.w);
            const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint32_t e = 4 * b + l;
                if (e >= e0 && e < e1) s_eps[e - e0] = z[l];
            }
        }
    } else {
        for (int i = lane; i < np_w * per; i += 32) s_eps[i] = pb.halton[static_cast<size_t>(nw0) * per + i];
    }
    __syncwarp();
    if (kFull && pb.filter != STORM_FILTER_DEFAULT) {  // comb-filtered particles, one sample per step (S = H)
        if (lane < np_w * d) {
            const int p = lane / d, j = lane - p * d;
            if (smoothing_of(pb, nw0 + p) == 2) comb_column(s_eps + p * S * d + j, H, d, pb.comb);
        }
        __syncwarp();
    }
    trace_stamp(pb.trace, 1);
    }
    // The noise depends on (seed, step, iteration) only, so under a dependent
    // launch it is drawn while the previous distribution update still runs;
    // mu and sigma are read after it has finished (from L2).
    if (kPhase != 2) pdl_wait();
    if (kPhase != 2 && pb.dep_launch) {  // the wait may have dropped the prefetched tables from L1
        const char* tb = reinterpret_cast<const char*>(pb.tables);
        for (int o = lane * 128; o < pb.table_bytes; o += 32 * 128)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(tb + o));
    }
    if (kPhase != 2 && do_costs) {
    if (pb.dep_launch)
        stage_inputs();  // after the previous update has finished
    else
        asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();

    // ---- controls u = mu + sigma o (B eps) of the lane's own steps, null particles zero
    for (int slot = 0; slot < W.SL; ++slot) {
        const int h = slot * Lp + hl;
        if (!pvalid || h >= H) continue;
        float e[kMaxDof];
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) e[j] = 0.f;
        if (smoothing_of(pb, n) == 1) {
            const float* eps = s_eps + seg * S * d;
            const int nk = pb.nk;
#pragma unroll 2
            for (int s = 0; s < nk; ++s) {
                const float b = s_basis[h * nk + s];
#pragma unroll
                for (int j = 0; j < kMaxDof; ++j)
                    if (j < d) e[j] = fmaf(b, eps[s * d + j], e[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kMaxDof; ++j)
                if (j < d) e[j] = s_eps[(seg * S + h) * d + j];
        }
        const bool null = n < pb.n_null;
        float* su = s_u + (seg * H + h) * d;
        float* gu = out.u + (static_cast<size_t>(n) * H + h) * d;
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            if (j < d) {
                const float uu = null ? 0.f : fmaf(s_sig[j], e[j], s_mu[h * d + j]);
                su[j] = uu;
                gu[j] = uu;
            }
        }
    }
    __syncwarp();
    // ---- integration per (particle, joint), Eq. 7: the k_rollout recurrence
    if (lane < np_w * d) {
        const int p = lane / d, j = lane - p * d;
        float v = s_st[d + j], q = s_st[j];
#pragma unroll 6
        for (int h = 0; h < H; ++h) {
            const int idx = (p * H + h) * d + j;
            v = fmaf(s_dt[h], s_u[idx], v);
            q = fmaf(s_dt[h], v, q);
            s_thd[idx] = v;
            s_th[idx] = q;
        }
    }
    __syncwarp();
    trace_stamp(pb.trace, 2);
    if (kFull && out.theta)
        for (int i = lane; i < np_w * HD; i += 32) out.theta[static_cast<size_t>(nw0) * HD + i] = s_th[i];
    if (kFull && out.theta_dot)
        for (int i = lane; i < np_w * HD; i += 32) out.theta_dot[static_cast<size_t>(nw0) * HD + i] = s_thd[i];
    }
    if (kPhase != 2 && kW > 1) unit_sync(unit, kW * 32);  // the other warps read the controls and joint states
    if (kPhase == 1) return;

    // ---- per-problem constants in registers
    int first[kMaxDof + 2];
#pragma unroll
    for (int f = 0; f < kMaxDof + 2; ++f) first[f] = f <= F ? pb.link_first[f] : pb.M;
    float4 lbf[kMaxDof + 1];
#pragma unroll
    for (int f = 0; f <= kMaxDof; ++f) lbf[f] = f < F ? pb.lbound[f] : make_float4(0.f, 0.f, 0.f, 0.f);
    float g[12] = {};  // goal rotation (row-major), then position (cost warp only)
    if (do_costs) {
        const float* goal = s_goal;
        const float qn = rsqrtf(goal[3] * goal[3] + goal[4] * goal[4] + goal[5] * goal[5] + goal[6] * goal[6]);
        const float w = goal[3] * qn, x = goal[4] * qn, y = goal[5] * qn, z = goal[6] * qn;
        g[0] = 1.f - 2.f * (y * y + z * z);
        g[1] = 2.f * (x * y - w * z);
        g[2] = 2.f * (x * z + w * y);
        g[3] = 2.f * (x * y + w * z);
        g[4] = 1.f - 2.f * (x * x + z * z);
        g[5] = 2.f * (y * z - w * x);
        g[6] = 2.f * (x * z - w * y);
        g[7] = 2.f * (y * z + w * x);
        g[8] = 1.f - 2.f * (x * x + y * y);
        g[9] = goal[0];
        g[10] = goal[1];
        g[11] = goal[2];
    }
    const bool want_manip = pb.w_manip != 0.f || (kFull && out.terms);
    const bool want_ee = kFull && (pb.w_ee_vel != 0.f || pb.w_ee_acc != 0.f || out.terms);
    const bool ball_on = kFull && pb.ball && pb.w_ball != 0.f;
    float* s_ba = ws + W.ba;
    const float* pred = (kFull || kPhase == 2) && pb.self_mode != 0 ? lane_pred : nullptr;
    const int NO = pb.B + pb.O;

    for (int slot = 0; slot < W.SL; ++slot) {
        const int h = slot * Lp + hl;
        const bool valid = pvalid && h < H;
        const int hc = valid ? h : 0;
        const int pl = pvalid ? seg : 0;
        const float* th = s_th + (pl * H + hc) * d;
        const float* thd = s_thd + (pl * H + hc) * d;
        const float* uh = s_u + (pl * H + hc) * d;
        const float* up = (hc == 0) ? s_st + 2 * d : uh - d;
        const size_t gi = static_cast<size_t>(n) * H + hc;  // global item (valid lanes)

        // ---- FK frames, Jacobian columns, bounding centres
        float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
        float pp[3] = {0.f, 0.f, 0.f};
        float J[6][kMaxDof];
        float oc[kMaxDof][3];  // joint origins (Eq. 8; the axes are J's angular rows)
        float cbx[kMaxDof + 1], cby[kMaxDof + 1], cbz[kMaxDof + 1];
        {
            const float fr0[12] = {1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f};
#pragma unroll
            for (int k = 0; k < 12; ++k) s_fr[k * 32 + lane] = fr0[k];
            cbx[0] = fmaf(1.f, lbf[0].x, fmaf(0.f, lbf[0].y, fmaf(0.f, lbf[0].z, 0.f)));
            cby[0] = fmaf(0.f, lbf[0].x, fmaf(1.f, lbf[0].y, fmaf(0.f, lbf[0].z, 0.f)));
            cbz[0] = fmaf(0.f, lbf[0].x, fmaf(0.f, lbf[0].y, fmaf(1.f, lbf[0].z, 0.f)));
        }
#pragma unroll
        for (int i = 0; i < kMaxDof; ++i) {
            if (i < d) {
                const float* dh = pb.dhx + i * 8;
                dh_step(R, pp, dh[0], dh[1], dh[2], dh[3], th[i] + dh[4]);
                {
                    float* fr = s_fr + (i + 1) * 12 * 32 + lane;
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        fr[(r * 4 + 0) * 32] = R[r * 3 + 0];
                        fr[(r * 4 + 1) * 32] = R[r * 3 + 1];
                        fr[(r * 4 + 2) * 32] = R[r * 3 + 2];
                        fr[(r * 4 + 3) * 32] = pp[r];
                    }
                }
                J[0][i] = pp[1] * R[8] - pp[2] * R[5];
                J[1][i] = pp[2] * R[2] - pp[0] * R[8];
                J[2][i] = pp[0] * R[5] - pp[1] * R[2];
                J[3][i] = R[2];
                J[4][i] = R[5];
                J[5][i] = R[8];
                oc[i][0] = pp[0], oc[i][1] = pp[1], oc[i][2] = pp[2];
                const float4 lb = lbf[i + 1];
                cbx[i + 1] = fmaf(R[0], lb.x, fmaf(R[1], lb.y, fmaf(R[2], lb.z, pp[0])));
                cby[i + 1] = fmaf(R[3], lb.x, fmaf(R[4], lb.y, fmaf(R[5], lb.z, pp[1])));
                cbz[i + 1] = fmaf(R[6], lb.x, fmaf(R[7], lb.y, fmaf(R[8], lb.z, pp[2])));
            } else {
#pragma unroll
                for (int r = 0; r < 6; ++r) J[r][i] = 0.f;
                oc[i][0] = oc[i][1] = oc[i][2] = 0.f;
                cbx[i + 1] = cby[i + 1] = cbz[i + 1] = 0.f;
            }
        }

        float part = 0.f;
        if (do_costs) {
        // pose (Eq. 9), rotation, stop (Eq. 10), joint limits (Eq. 11), smoothness
        const float dx = pp[0] - g[9], dy = pp[1] - g[10], dz = pp[2] - g[11];
        float c_pos = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float e = pb.pos_w[a] * fmaf(g[a], dx, fmaf(g[3 + a], dy, g[6 + a] * dz));
            c_pos = fmaf(e, e, c_pos);
        }
        c_pos = sqrtf(c_pos);
        float c_rot = 0.f;
        if (!kFull || pb.rot_mode == STORM_ROT_QUAT) {
            float tr = 0.f;
#pragma unroll
            for (int k = 0; k < 9; ++k) tr = fmaf(g[k], R[k], tr);
            c_rot = 1.f - 0.5f * sqrtf(fmaxf(0.f, 1.f + tr));
        } else {
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float rtr = fmaf(g[r], R[c], fmaf(g[3 + r], R[3 + c], g[6 + r] * R[6 + c]));
                    const float e = ((r == c) ? 1.f : 0.f) - rtr;
                    const float we = e * pb.rot_w[c];
                    c_rot = fmaf(we, we, c_rot);
                }
            c_rot = sqrtf(c_rot);
        }
        float c_stop = 0.f, c_joint = 0.f, c_smooth = 0.f;
        const float vlim = pb.vmax[hc];
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            if (j < d) {
                const float vs = fmaxf(0.f, fabsf(thd[j]) - vlim);
                c_stop = fmaf(vs, vs, c_stop);
                const float vj = fmaxf(0.f, pb.qlo[j] - th[j]) + fmaxf(0.f, th[j] - pb.qhi[j]);
                c_joint = fmaf(vj, vj, c_joint);
                const float du = uh[j] - up[j];
                c_smooth = fmaf(du, du, c_smooth);
            }
        }
        c_stop = sqrtf(c_stop);
        c_joint = sqrtf(c_joint);
        part = pb.w_pos * c_pos + pb.w_rot * c_rot + pb.w_stop * c_stop + pb.w_joint * c_joint +
               pb.w_smooth * c_smooth;
        float2 c_ee = make_float2(0.f, 0.f);
        if (want_ee) {  // task-space limits on X_dot, X_ddot (Eq. 8), theta_ddot = u
            float zc[kMaxDof][3];
#pragma unroll
            for (int i = 0; i < kMaxDof; ++i) zc[i][0] = J[3][i], zc[i][1] = J[4][i], zc[i][2] = J[5][i];
            float xd[6], xdd[6];
            ee_twist(zc, oc, pp, thd, uh, d, xd, xdd);
            c_ee = ee_limit_terms(pb, xd, xdd);
            if (pb.w_ee_vel != 0.f) part = fmaf(pb.w_ee_vel, c_ee.x, part);
            if (pb.w_ee_acc != 0.f) part = fmaf(pb.w_ee_acc, c_ee.y, part);
        }
        if (ball_on && valid) {
            const float2 a = ball_accel(R, pb.grav);
            s_ba[(pl * H + h) * 2] = a.x;
            s_ba[(pl * H + h) * 2 + 1] = a.y;
        }
        if (kFull && valid && out.ee) {
            float* e = out.ee + gi * 12;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                e[r * 4 + 0] = R[r * 3 + 0];
                e[r * 4 + 1] = R[r * 3 + 1];
                e[r * 4 + 2] = R[r * 3 + 2];
                e[r * 4 + 3] = pp[r];
            }
        }
        if (kFull && valid && out.terms) {
            float* t = out.terms + gi * STORM_NTERMS;
            t[0] = c_pos;
            t[1] = c_rot;
            t[2] = c_stop;
            t[3] = c_joint;
            t[7] = c_smooth;
            t[8] = c_ee.x;
            t[9] = c_ee.y;
            t[10] = 0.f;
        }
        }  // do_costs
        // manipulability (Eq. 12)
        float c_manip = 0.f;
        if (do_manipw && want_manip) {
            const float m = manipulability_mgs(J, d);
            c_manip = (m < pb.k_m) ? 1.f - m : 0.f;
            if (kW == 1) part += pb.w_manip * c_manip;  // pair and quad: A adds it at the hand-off
            if (kFull && valid && out.terms) out.terms[gi * STORM_NTERMS + 4] = c_manip;
        }
        __syncwarp();
        trace_stamp(pb.trace, 3);

        // ---- world collision, Eq. 14 reading
        float dworld = 0.f;
        if (do_world && NO > 0 && pb.M > 0) {
            if (pb.broadphase) {
                // box enclosing every link bound of the warp's items, padded 1 mm
                float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
                for (int f = 0; f <= kMaxDof; ++f) {
                    if (f < F && valid && first[f] < first[f + 1]) {
                        const float r = lbf[f].w + 1e-3f;
                        lo[0] = fminf(lo[0], cbx[f] - r);
                        lo[1] = fminf(lo[1], cby[f] - r);
                        lo[2] = fminf(lo[2], cbz[f] - r);
                        hi[0] = fmaxf(hi[0], cbx[f] + r);
                        hi[1] = fmaxf(hi[1], cby[f] + r);
                        hi[2] = fmaxf(hi[2], cbz[f] + r);
                    }
                }
                // the lane's own box (its item's link bounds), kept before the warp's union
                const float llo0 = lo[0], llo1 = lo[1], llo2 = lo[2], lhi0 = hi[0], lhi1 = hi[1], lhi2 = hi[2];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = fminf(lo[a], __shfl_xor_sync(FULL, lo[a], o));
                        hi[a] = fmaxf(hi[a], __shfl_xor_sync(FULL, hi[a], o));
                    }
                }
                for (int k0 = 0; k0 < NO; k0 += 32) {
                    const int k = k0 + lane;
                    bool near = false;
                    if (k < pb.B) {
                        const float* b = pb.boxes + k * 6;
                        near = b[0] - b[3] <= hi[0] && b[0] + b[3] >= lo[0] && b[1] - b[4] <= hi[1] &&
                               b[1] + b[4] >= lo[1] && b[2] - b[5] <= hi[2] && b[2] + b[5] >= lo[2];
                    } else if (k < NO) {
                        const float4 w = pb.wsph[k - pb.B];
                        const float ex = w.x - fminf(fmaxf(w.x, lo[0]), hi[0]);
                        const float ey = w.y - fminf(fmaxf(w.y, lo[1]), hi[1]);
                        const float ez = w.z - fminf(fmaxf(w.z, lo[2]), hi[2]);
                        near = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= w.w * w.w;
                    }
                    unsigned mask = __ballot_sync(FULL, near);
                    while (mask) {
                        const int kk = k0 + __ffs(mask) - 1;
                        mask &= mask - 1;
                        if (!valid) continue;
                        if (kk < pb.B) {
                            const float* box = pb.boxes + kk * 6;
                            const float lox = box[0] - box[3], loy = box[1] - box[4], loz = box[2] - box[5];
                            const float hix = box[0] + box[3], hiy = box[1] + box[4], hiz = box[2] + box[5];
                            // clear of the lane's box: no link bound of the item meets the box
                            if (!(lox <= lhi0 && hix >= llo0 && loy <= lhi1 && hiy >= llo1 && loz <= lhi2 &&
                                  hiz >= llo2))
                                continue;
                            unsigned fm = 0u;  // the frames whose bound meets the box
#pragma unroll
                            for (int f = 0; f <= kMaxDof; ++f) {
                                if (f < F && first[f] < first[f + 1]) {
                                    const float ex = cbx[f] - fminf(fmaxf(cbx[f], lox), hix);
                                    const float ey = cby[f] - fminf(fmaxf(cby[f], loy), hiy);
                                    const float ez = cbz[f] - fminf(fmaxf(cbz[f], loz), hiz);
                                    if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < lbf[f].w * lbf[f].w) fm |= 1u << f;
                                }
                            }
                            // each lane its own frames, the lanes side by side (depths combine by max:
                            // any order gives the same bits)
                            while (fm) {
                                const int f = __ffs(fm) - 1;
                                fm &= fm - 1u;
                                int s0 = 0, s1 = 0;
#pragma unroll
                                for (int g = 0; g <= kMaxDof; ++g)
                                    if (g == f) s0 = first[g], s1 = first[g + 1];
                                dworld = box_depth(s_fr + f * 12 * 32, lane, pb.sph, s0, s1, box, dworld);
                            }
                        } else {
                            const float4 w = pb.wsph[kk - pb.B];
                            {  // clear of the lane's box: no link bound of the item reaches the ball
                                const float ex = w.x - fminf(fmaxf(w.x, llo0), lhi0);
                                const float ey = w.y - fminf(fmaxf(w.y, llo1), lhi1);
                                const float ez = w.z - fminf(fmaxf(w.z, llo2), lhi2);
                                if (!(fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= w.w * w.w)) continue;
                            }
                            unsigned fm = 0u;
#pragma unroll
                            for (int f = 0; f <= kMaxDof; ++f) {
                                if (f < F && first[f] < first[f + 1]) {
                                    const float ex = cbx[f] - w.x, ey = cby[f] - w.y, ez = cbz[f] - w.z;
                                    const float rb = lbf[f].w + w.w;
                                    if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rb * rb) fm |= 1u << f;
                                }
                            }
                            while (fm) {
                                const int f = __ffs(fm) - 1;
                                fm &= fm - 1u;
                                int s0 = 0, s1 = 0;
#pragma unroll
                                for (int g = 0; g <= kMaxDof; ++g)
                                    if (g == f) s0 = first[g], s1 = first[g + 1];
                                dworld = ball_depth(s_fr + f * 12 * 32, lane, pb.sph, s0, s1, w, dworld);
                            }
                        }
                    }
                }
            } else if (valid) {
                dworld = world_brute_force(s_fr, lane, pb.link_first, pb.sph, F, pb.boxes, pb.B, pb.wsph, pb.O,
                                           dworld);
            }
        }
        trace_stamp(pb.trace, 4);

        // ---- self collision, Eq. 13 reading: frame pairs whose bounding
        // spheres overlap (register tests over the compile-time list of pairs)
        // and whose capsules meet, then their pair blocks exactly, each
        // first-frame sphere first tested against the second frame's capsule;
        // then the leftover pairs
        float dself = 0.f;
        const float pv = pred && valid ? pred[slot * kMlpRows] : 0.f;
        const bool do_self = do_selfc && valid && !(pred && (pb.self_mode == 2 || pv >= pb.self_margin));
        if (valid && pred && pb.self_mode == 2) dself = fmaxf(0.f, pv);  // Eq. 13's learned term
        uint32_t lp_hit = 0u;  // bit t: frame pair t has blocks and its bounds overlap
        // pair: B publishes the item's mask, then works from its first pair, A
        // from its last; each announces a pair before testing it and stops where
        // the other has announced.  A stale read only repeats a test (the depth
        // is a max), never skips one.  A joins only where B's mask is published
        // (bit 31) by the time A's own terms are done.
        static_assert(kLinkPairs <= 31, "bit 31 of a published mask marks it published");
        int hit_no = 0;  // the quad's C and D take alternate hits of each lane
        volatile int* item = reinterpret_cast<volatile int*>(ws + W.claim) + slot * 32 + lane;
        volatile int* started_b = item + W.SL * 32;
        volatile int* started_a = item + 2 * W.SL * 32;
        const bool joins = kW == 2 && do_costs;  // the pair's A
        if (kW == 2 && joins) __syncwarp();  // (A's read stays after its own terms)
        if (joins && do_self) {
            uint32_t m;
            asm volatile("ld.volatile.shared.u32 %0, [%1];"
                         : "=r"(m)
                         : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(const_cast<int*>(item))))
                         : "memory");
            lp_hit = (m >> 31) ? (m & 0x7fffffffu) : 0u;
        }
        if (do_self && !joins) {
#pragma unroll
            for (int la = 0; la < kMaxDof; ++la) {
#pragma unroll
                for (int lb = la + 1; lb <= kMaxDof; ++lb) {
                    const int t = link_pair_index(la, lb);
                    if (lb < F && pb.lp_begin[t] < pb.lp_begin[t + 1]) {
                        bool pass = true;
                        if (pb.broadphase) {
                            const float ex = cbx[la] - cbx[lb], ey = cby[la] - cby[lb], ez = cbz[la] - cbz[lb];
                            const float rr = lbf[la].w + lbf[lb].w;
                            pass = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rr * rr;
                        }
                        if (pass) lp_hit |= 1u << t;
                    }
                }
            }
            if (pb.broadphase) {  // of those, the frame pairs whose capsules meet too
                uint32_t m = lp_hit;
                while (m) {
                    const int t = __ffs(m) - 1;
                    m &= m - 1;
                    int la = 0;  // t = link_pair_index(la, lk)
#pragma unroll
                    for (int f = 1; f < kMaxDof; ++f) la += t >= link_pair_index(f, f + 1);
                    const int lk = t - link_pair_index(la, la + 1) + la + 1;
                    const float4 a0 = pb.lcap[2 * la], a1 = pb.lcap[2 * la + 1];
                    const float4 b0 = pb.lcap[2 * lk], b1 = pb.lcap[2 * lk + 1];
                    const float* fa = s_fr + la * 12 * 32;
                    const float* fb = s_fr + lk * 12 * 32;
                    const float rr = a0.w + b0.w;
                    if (seg_seg_dist2(frame_point(fa, lane, a0), frame_point(fa, lane, a1), frame_point(fb, lane, b0),
                                      frame_point(fb, lane, b1)) >= rr * rr)
                        lp_hit &= ~(1u << t);
                }
            }
        }
        if (kW == 2 && do_self && !joins) *item = static_cast<int>(lp_hit | 0x80000000u);
        const int n_hit = __popc(lp_hit);
        int taken = 0;  // pairs this warp has started
        while (lp_hit) {
            int t;
            if (kW == 2) {
                if (joins) {
                    if (n_hit - 1 - taken < *started_b) break;
                    t = 31 - __clz(lp_hit);
                    *started_a = ++taken;
                } else {
                    if (taken >= n_hit - *started_a) break;
                    t = __ffs(lp_hit) - 1;
                    *started_b = ++taken;
                }
                lp_hit &= ~(1u << t);
            } else {
                t = __ffs(lp_hit) - 1;
                lp_hit &= lp_hit - 1;
                if (self_half >= 0 && (hit_no++ & 1) != self_half) continue;
            }
            const int* lpb = reinterpret_cast<const int*>(ws + W.lpb);
            const int bk0 = lpb[t], bk1 = lpb[t + 1];  // the pair's blocks: spheres of frame la x frame lk
            int la = 0;  // t = link_pair_index(la, lk)
#pragma unroll
            for (int f = 1; f < kMaxDof; ++f) la += t >= link_pair_index(f, f + 1);
            const int lk = t - link_pair_index(la, la + 1) + la + 1;
            // the second frame's capsule: the segment k0 + s ke, s in [0, 1], radius kc0.w
            const float4 kc0 = pb.lcap[2 * lk], kc1 = pb.lcap[2 * lk + 1];
            const float3 k0 = frame_point(s_fr + lk * 12 * 32, lane, kc0);
            const float3 k1 = frame_point(s_fr + lk * 12 * 32, lane, kc1);
            const float3 ke = make_float3(k1.x - k0.x, k1.y - k0.y, k1.z - k0.z);
            const float kee = fmaf(ke.x, ke.x, fmaf(ke.y, ke.y, ke.z * ke.z));
            const float kinv = kee > 1e-12f ? __frcp_rn(kee) : 0.f;
            float fa[12];  // the first frame, for every sphere of its blocks
#pragma unroll
            for (int k = 0; k < 12; ++k) fa[k] = s_fr[(la * 12 + k) * 32 + lane];
            const float* fb = s_fr + lk * 12 * 32;
            for (int bk = bk0; bk < bk1; ++bk) {
                const uint4 blk = pb.pblk[bk];  // a0, a1, b0, nb
                // second-frame spheres in pairs (k, k + 4) for the packed tests: negated
                // centre coordinates and radii
                float2 nbx[4], nby[4], nbz[4], rb[4];
                bool have_b = false;  // second-frame centres, computed on first need
                for (uint32_t a = blk.x; a < blk.y; ++a) {
                    const float4 q = pb.sph[a];
                    const float3 c = make_float3(fmaf(fa[0], q.x, fmaf(fa[1], q.y, fmaf(fa[2], q.z, fa[3]))),
                                                 fmaf(fa[4], q.x, fmaf(fa[5], q.y, fmaf(fa[6], q.z, fa[7]))),
                                                 fmaf(fa[8], q.x, fmaf(fa[9], q.y, fmaf(fa[10], q.z, fa[11]))));
                    if (pb.broadphase) {  // sphere a apart from the second frame's capsule: no pair touches
                        const float dx = c.x - k0.x, dy = c.y - k0.y, dz = c.z - k0.z;
                        const float sp = clamp01(fmaf(dx, ke.x, fmaf(dy, ke.y, dz * ke.z)) * kinv);
                        const float ex = fmaf(-sp, ke.x, dx), ey = fmaf(-sp, ke.y, dy), ez = fmaf(-sp, ke.z, dz);
                        const float rr = q.w + kc0.w;
                        if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) >= rr * rr) continue;
                    }
                    if (!have_b) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            float4 cb4 = make_float4(-1e30f, -1e30f, -1e30f, 0.f);
                            if (k < static_cast<int>(blk.w)) {
                                const float4 qb = pb.sph[blk.z + k];
                                const float3 cb = frame_point(fb, lane, qb);
                                cb4 = make_float4(-cb.x, -cb.y, -cb.z, qb.w);
                            }
                            if (k < 4) {
                                nbx[k].x = cb4.x, nby[k].x = cb4.y, nbz[k].x = cb4.z, rb[k].x = cb4.w;
                            } else {
                                nbx[k - 4].y = cb4.x, nby[k - 4].y = cb4.y, nbz[k - 4].y = cb4.z, rb[k - 4].y = cb4.w;
                            }
                        }
                        have_b = true;
                    }
                    // the exact tests two at a time (Blackwell's paired FP32 operations:
                    // per half the same IEEE operations in the same order as one test)
                    const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y),
                                 cz = make_float2(c.z, c.z), qw = make_float2(q.w, q.w);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 ex = __fadd2_rn(cx, nbx[k]), ey = __fadd2_rn(cy, nby[k]),
                                     ez = __fadd2_rn(cz, nbz[k]);
                        const float2 dist2 = __ffma2_rn(ex, ex, __ffma2_rn(ey, ey, __fmul2_rn(ez, ez)));
                        const float2 rs = __fadd2_rn(qw, rb[k]);
                        const float2 rr = __fmul2_rn(rs, rs);
                        if (dist2.x < rr.x) dself = fmaxf(dself, rs.x - sqrtf(dist2.x));
                        if (dist2.y < rr.y) dself = fmaxf(dself, rs.y - sqrtf(dist2.y));
                    }
                }
            }
        }
        if (do_self && !(kW == 2 && do_costs)) {  // the leftover pairs: not the pair's A
            for (int k = self_half > 0 ? 1 : 0; k < pb.P; k += self_half >= 0 ? 2 : 1) {
                const uint32_t pr = pb.pairs[k];
                const int a = pr & 0xffff, b = pr >> 16;
                int la = 0, lk = 0;
#pragma unroll
                for (int f = 1; f <= kMaxDof; ++f) {
                    if (f <= d) {
                        la += a >= first[f];
                        lk += b >= first[f];
                    }
                }
                const float4 qa = pb.sph[a], qb = pb.sph[b];
                const float rs = qa.w + qb.w;
                const float3 ca = frame_point(s_fr + la * 12 * 32, lane, qa);
                const float3 cb = frame_point(s_fr + lk * 12 * 32, lane, qb);
                const float ex = ca.x - cb.x, ey = ca.y - cb.y, ez = ca.z - cb.z;
                const float dist2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                if (dist2 < rs * rs) dself = fmaxf(dself, rs - sqrtf(dist2));
            }
        }
        trace_stamp(pb.trace, 5);

        // ---- running cost (Eq. 15)
        if (kW > 1) {  // the other warps hand their results to A
            float* hand = ws + W.hand;
            const int PH = W.PW * H, ix = pl * H + h;
            if (valid) {
                if (do_selfc && !do_costs) hand[(self_half > 0 ? PH : 0) + ix] = dself;
                if (kW == 4 && do_world) hand[2 * PH + ix] = dworld;
                if (do_manipw) hand[3 * PH + ix] = c_manip;
            }
            unit_sync(unit, kW * 32);
            if (do_costs && valid) {
                if (want_manip) part += pb.w_manip * hand[3 * PH + ix];  // the single-warp order
                if (kW == 2) {
                    dself = fmaxf(dself, hand[ix]);  // A's own pairs, then B's
                } else {
                    dself = fmaxf(hand[ix], hand[PH + ix]);
                    dworld = hand[2 * PH + ix];
                }
            }
        }
        if (do_costs) {
            const float c = part + pb.w_coll * (dself + dworld);
            if (valid) {
                s_c[pl * H + h] = c;
                if (kFull && out.terms) {
                    out.terms[gi * STORM_NTERMS + 5] = dself;
                    out.terms[gi * STORM_NTERMS + 6] = dworld;
                }
            }
        }
        __syncwarp();  // the next slot rewrites the frames
    }
    if (!do_costs) return;  // B is done
    if (ball_on) {  // the ball along each particle's horizon
        if (lane < np_w) {
            ball_tail(pb.dhx, d, state, pb.ball, H, pb.w_ball, pb.tray[0], pb.tray[1], s_ba + lane * H * 2, pb.dt,
                      s_c + lane * H,
                      out.terms ? out.terms + (static_cast<size_t>(nw0 + lane) * H) * STORM_NTERMS + 10 : nullptr);
        }
        __syncwarp();
    }
    if (kFull && out.cost)
        for (int slot = 0; slot < W.SL; ++slot) {
            const int h = slot * Lp + hl;
            if (pvalid && h < H) out.cost[static_cast<size_t>(n) * H + h] = s_c[seg * H + h];
        }
    // ---- discounted total (Eq. 2), the k_rollout order
    if (lane < np_w) {
        float C = 0.f;
#pragma unroll 6
        for (int h = 0; h < H; ++h) C = fmaf(s_gp[h], s_c[lane * H + h], C);
        out.Ctot[nw0 + lane] = C;
    }
    trace_stamp(pb.trace, 6);
}

template <int kW, bool kFull>
__global__ void __launch_bounds__(kWarpMaxWarps * 32, 1)
k_rollout_warp(Problem pb, RolloutOut out, const float* __restrict__ state, const float* __restrict__ goal,
               const StepState* __restrict__ st, int step_override, int iter)
{
    extern __shared__ __align__(16) float wsm[];
    const WarpPlan W = warp_plan(pb, kW);
    const int warp = threadIdx.x >> 5;
    const int unit = warp / kW;  // the kW warps of a particle group
    const int units = (blockDim.x >> 5) / kW;
    pdl_trigger();
    const uint32_t step = step_override >= 0 ? static_cast<uint32_t>(step_override) : st->step;
    rollout_warp_body<kW, kFull>(pb, out, state, goal, step, iter, blockIdx.x * units + unit, unit,
                             wsm + unit * W.floats);
}
