// storm_rollout_mlp.cuh -- generate_rollouts with the learned self-collision
// network (Sec. 4.2, Eq. 13) evaluated inside the rollout kernel.
//
// One CTA of six warps: four take warp-mapped particle groups (one particle per
// warp for H > 16), so that each item slot of theirs is one 128-row tile of the
// network (row 32 w + lane is warp w's lane), and drain the tensor core's
// accumulators; the fifth issues the MMAs; the sixth keeps the weights
// streaming.  The warps first draw the
// noise, form the controls and integrate them (Eq. 7) exactly as the warp
// mapping does; then the CTA encodes each row's joint state into shared memory
// and runs the whole network on the tile on the tensor cores
// (tc::mlp_tile_forward: BF16 operands, FP32 accumulation in TMEM, weights
// streamed by bulk asynchronous copies -- the first blocks already in flight
// while the noise is drawn); then each warp finishes its items (FK, Jacobian, costs,
// world collision) and runs the exact self-collision check only where the
// prediction asks for it: below the margin (gate), or never (the learned cost
// max(0, prediction)).  The exact check is also the fallback: if a
// tensor-core wait runs out, the CTA sets the network's error flag and every
// item of the CTA takes the exact check.
#pragma once

constexpr int kMlpWarps = kMlpRows / 32;  // one warp per 32 rows of a tile

// Shared-memory plan of a k_rollout_mlp CTA (bytes): the network's tile
// (ring | activations | vectors), the predictions of every item slot, then
// the four warps' rollout regions.
struct MlpRolloutPlan {
    int pred;   // SL x 128 floats
    int roll;   // 4 x WarpPlan::floats floats
    int bytes;
};

__host__ __device__ inline MlpRolloutPlan mlp_rollout_plan(const Problem& pb)
{
    const WarpPlan W = warp_plan(pb, 1);
    MlpRolloutPlan P;
    P.pred = static_cast<int>(tc::kTileSmem);
    P.roll = P.pred + W.SL * kMlpRows * 4;
    P.bytes = P.roll + kMlpWarps * W.floats * 4;
    return P;
}

constexpr int kMlpEpi = kMlpWarps;  // the rolling warps are the network's epilogue warps

// kFull: as for k_rollout_warp (the lean instantiation when the problem and the
// call need nothing beyond the default path and the network).
template <bool kFull>
__global__ void __launch_bounds__(tc::tile_threads(kMlpEpi), 1)
k_rollout_mlp(Problem pb, RolloutOut out, const float* __restrict__ state, const float* __restrict__ goal,
              const StepState* __restrict__ st, int step_override, int iter, tc::MlpView net)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];
    __shared__ __align__(8) uint64_t bars[tc::kTileBars];
    __shared__ uint32_t tmem_slot;
    unsigned char* smem = tile_smem;
    const WarpPlan W = warp_plan(pb, 1);
    const MlpRolloutPlan P = mlp_rollout_plan(pb);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool roller = warp < kMlpWarps;  // warps 0-3 roll out; warp 4 issues the MMAs, warp 5 the copies
    const uint32_t step = step_override >= 0 ? static_cast<uint32_t>(step_override) : st->step;
    float* ws = reinterpret_cast<float*>(smem + P.roll) + (roller ? warp : 0) * W.floats;
    float* s_pred = reinterpret_cast<float*>(smem + P.pred);
    float* s_b2 = reinterpret_cast<float*>(smem + tc::kOffVec);
    float* s_b3 = s_b2 + 256;
    float* s_w4 = s_b3 + 256;
    float* s_part = s_w4 + 256;
    const int wg = blockIdx.x * kMlpWarps + (roller ? warp : 0);

    // the first weight blocks land while the noise is drawn
    tc::MlpTiles t;
    tc::mlp_tiles_init<kMlpEpi>(t, net, tc::smem_u32(smem), bars, &tmem_slot, W.SL * tc::mlp_blocks(net));
    for (int n = tid; n < 256; n += blockDim.x) {
        s_b2[n] = n < net.h2 ? net.b2[n] : 0.f;
        s_b3[n] = n < net.h3 ? net.b3[n] : 0.f;
        s_w4[n] = n < net.h3 ? net.w4[n] : 0.f;
    }
    const float b4 = *net.b4;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    t.tmem = tmem_slot;

    // ---- noise, controls, integration (Eq. 7): each rolling warp's joint states in its region
    if (roller) rollout_warp_body<1, kFull, 1>(pb, out, state, goal, step, iter, wg, warp, ws);
    __syncwarp();

    // ---- the network on every item slot's tile (row 32 w + lane = rolling warp w's lane)
    const int Lp = W.Lp, seg = lane / Lp, hl = lane - seg * Lp;
    const int n0 = wg * W.PW;
    const int np_w = n0 < pb.N ? min(W.PW, pb.N - n0) : 0;
    bool ok = true;
    for (int slot = 0; slot < W.SL && ok; ++slot) {
        bool mine = true;
        if (roller) {
            const int h = slot * Lp + hl;
            float in[kMlpIn];
            if (seg < np_w && h < pb.H) {
                mlp_encode_row(ws + W.th + (seg * pb.H + h) * pb.d, pb.d, net.enc, in);
            } else {
#pragma unroll
                for (int i = 0; i < kMlpIn; ++i) in[i] = 0.f;
            }
            mlp_store_input_row(t.sA1, tid, in);
            tc::mlp_announce(tc::tile_a1(t));
            float y = 0.f;
            mine = tc::mlp_tile_epilogue<kMlpEpi>(net, t, s_b2, s_b3, s_w4, s_part, b4, &y);
            s_pred[slot * kMlpRows + tid] = y;
        } else if (warp == kMlpEpi && lane == 0) {
            mine = tc::mlp_tile_issue(net, t);
        } else if (warp == kMlpEpi + 1 && lane == 0) {
            mine = tc::mlp_load_all(net, t, (slot + 1) * tc::mlp_blocks(net));  // this slot's weight blocks
        }
        ok = __syncthreads_and(mine);  // the same decision on every thread
    }
    if (!ok) {
        if (tid == kMlpEpi * 32) {
            if (net.err) atomicExch(net.err, 1);
            tc::mlp_drain_mmas(t);
        } else if (tid == (kMlpEpi + 1) * 32) {
            tc::mlp_drain_loads(t);
        }
        __syncthreads();
    }

    // ---- the rest of the rollout, the exact self check where the prediction asks for it
    if (roller)
        rollout_warp_body<1, kFull, 2>(pb, out, state, goal, step, iter, wg, warp, ws, ok ? s_pred + tid : nullptr);

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(tc::kTileCols) : "memory");
}
