// Krylov-loop pass 1 of the mixed-precision inner solves on the 5th-generation tensor cores
// (tcgen05, kind::tf32, accumulators in tensor memory).
//
// Per element e the pass is the complex product [x_E; t_T] = W r_E with W = [S_E^-1; Y^T]
// ((n_E + n_T) x n_E, formed at factor time; Sec. 2.3.3, eq. block_matrix_inversion with the
// explicit edge operators) and r_E the element's type-1 edge values of C1^T z for a block of
// right-hand sides.  In real arithmetic
//     Re x = Wr Rr - Wi Ri,   Im x = Wr Ri + Wi Rr,
// four real MMAs per K-step of 8 (the second with the A operand negated), accumulated in two
// TMEM accumulators of M = 128 lanes x NB columns.
//
// Operands live in shared memory in the no-swizzle K-major canonical layout: core matrices of
// 8 rows x 16 bytes (4 tf32), the core matrix of (row group g, column group c) at
// g * SBO + c * 128 bytes, SBO = (Kp / 4) * 128.  W's real and imaginary planes are stored in
// exactly this layout at factor time, so one bulk copy (cp.async.bulk) stages an element; the
// right-hand sides are gathered from the FP64 dual vector, converted and written by the CTA's
// threads.  One persistent launch walks the elements in the order of `items` (degree
// descending, so the heavy elements start first); the next element's W copy is issued as soon
// as the current element's MMAs have completed.  Rows of the 128-lane accumulator beyond the
// element's n_E + n_T come from whatever the staging buffer holds and are never written out.
#include "ddh_kcommon.cuh"

namespace ddh {

namespace {

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;               // leading byte offset: next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;     // stride byte offset: next group of 8 rows
    d |= (uint64_t)1 << 46;                         // descriptor version (tcgen05)
    return d;                                       // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = NB
__device__ __forceinline__ uint32_t umma_idesc(int NB, bool negA) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (negA ? (1u << 13) : 0u) | ((uint32_t)(NB >> 3) << 17) |
           ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dt), "l"(a), "l"(b), "r"(idesc),
                 "r"((uint32_t)acc)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__host__ __device__ __forceinline__ int round8(int x) { return (x + 7) & ~7; }

// round to the nearest tf32 (10-bit mantissa), kept in an fp32 container
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace

// floats of one W plane of an element with n_E type-1 edge and n_T type-2 slots
__host__ __device__ inline int64_t tc_plane_floats(int nE, int nT) {
    return (int64_t)((nE + nT + 7) / 8) * (((nE + 7) & ~7) / 4) * 32;
}

template <int NB>
__global__ void __launch_bounds__(128, 1) k_pass1_tc(DevModel dm, const float* __restrict__ W,
                                                     const int64_t* __restrict__ w_off, const int* __restrict__ items,
                                                     int n_items, const double2* __restrict__ z, double zsign, int R,
                                                     cpx<float>* __restrict__ xE_out, cpx<float>* __restrict__ tT_out,
                                                     const int* __restrict__ done, int a_bytes) {
    if (done && *done) return;
    extern __shared__ __align__(1024) char smem[];
    uint64_t* bar_a = reinterpret_cast<uint64_t*>(smem);
    uint64_t* bar_m = reinterpret_cast<uint64_t*>(smem + 8);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
    int* fail = reinterpret_cast<int*>(smem + 20);
    float* sA = reinterpret_cast<float*>(smem + 1024);
    float* sB = reinterpret_cast<float*>(smem + 1024 + a_bytes);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    constexpr uint32_t kCols = NB * 2 < 32 ? 32 : NB * 2;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_a)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar_m)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tmem_slot;
    const uint32_t tre = tbase, tim = tbase + NB;
    uint32_t ph_a = 0, ph_m = 0;
    // W of the first element in flight
    auto issue_a = [&](int item) {
        const int e = items[item];
        const int nE = dm.nE1[e], nT = dm.nT[e];
        if (nE == 0) return false;
        const uint32_t bytes = (uint32_t)(2 * tc_plane_floats(nE, nT) * sizeof(float));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar_a)), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(sA)), "l"(W + w_off[e]), "r"(bytes), "r"(smem_u32(bar_a))
                     : "memory");
        return true;
    };
    bool a_pending = false;
    if (t == 0 && blockIdx.x < n_items) a_pending = issue_a(blockIdx.x);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int e = items[item];
        const int nE = dm.nE1[e], nT = dm.nT[e], e1o = dm.e1_off[e], to = dm.t_off[e];
        const int M = nE + nT, Kp = round8(nE);
        const uint32_t sbo = (uint32_t)(Kp / 4) * 128u;
        const int64_t pf = tc_plane_floats(nE, nT);
        const int64_t bpf = (int64_t)(NB / 8) * (Kp / 4) * 32;       // floats of one B plane
        const int next = item + gridDim.x;
        for (int r0 = 0; r0 < R; r0 += NB) {
            const int cnt = min(NB, R - r0);
            if (nE == 0) {
                // no edge unknowns: t_T = Y^T r_E = 0
                for (int idx = t; idx < cnt * nT; idx += blockDim.x) {
                    const int q = idx / nT, o = idx % nT;
                    tT_out[(int64_t)(r0 + q) * dm.nT_tot + to + o] = mk<float>(0.f, 0.f);
                }
                continue;
            }
            // right-hand sides: B[q][j] = zsign * sign_j * z[r0+q][row_j] (tf32), zero padded
            for (int idx = t; idx < NB * Kp; idx += blockDim.x) {
                const int q = idx / Kp, j = idx % Kp;
                float vr = 0.f, vi = 0.f;
                if (q < cnt && j < nE) {
                    const int row = dm.e1_row[e1o + j];
                    if (row >= 0) {
                        const double s = zsign * dm.e1_sign[e1o + j];
                        const double2 v = z[(int64_t)(r0 + q) * dm.n_dual + row];
                        vr = to_tf32((float)(s * v.x));
                        vi = to_tf32((float)(s * v.y));
                    }
                }
                const int off = ((q >> 3) * (Kp / 4) + (j >> 2)) * 32 + (q & 7) * 4 + (j & 3);
                sB[off] = vr;
                sB[bpf + off] = vi;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (t == 0) {
                bool ok = true;
                if (a_pending) {
                    ok = mbar_wait_bounded(bar_a, ph_a);
                    ph_a ^= 1;
                    a_pending = false;
                }
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t aR = smem_u32(sA), aI = smem_u32(sA + pf);
                    const uint32_t bR = smem_u32(sB), bI = smem_u32(sB + bpf);
                    const uint32_t ipos = umma_idesc(NB, false), ineg = umma_idesc(NB, true);
                    for (int ks = 0; ks < Kp / 8; ++ks) {
                        const uint32_t adv = (uint32_t)ks * 256u;
                        umma(tre, umma_desc(aR + adv, sbo), umma_desc(bR + adv, sbo), ipos, ks > 0);
                        umma(tre, umma_desc(aI + adv, sbo), umma_desc(bI + adv, sbo), ineg, true);
                        umma(tim, umma_desc(aR + adv, sbo), umma_desc(bI + adv, sbo), ipos, ks > 0);
                        umma(tim, umma_desc(aI + adv, sbo), umma_desc(bR + adv, sbo), ipos, true);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(smem_u32(bar_m)) : "memory");
                    ok = mbar_wait_bounded(bar_m, ph_m);
                    ph_m ^= 1;
                }
                if (!ok) {
                    *fail = 1;
                    if (dm.err) atomicExch(dm.err, 4);
                } else if (r0 + NB >= R && next < n_items) {
                    // this element's MMAs have read W: start the next element's copy
                    a_pending = issue_a(next);
                }
            }
            __syncthreads();
            if (*fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // epilogue: TMEM lane o (warp w reads lanes 32w .. 32w+31) is output row o
            const int o = warp * 32 + lane;
            const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
#pragma unroll
            for (int c0 = 0; c0 < NB; c0 += 16) {
                float vr[16], vi[16];
                tmem_ld16(tre + lanebase + c0, vr);
                tmem_ld16(tim + lanebase + c0, vi);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (o < M)
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int q = c0 + i;
                        if (q < cnt) {
                            if (o < nE) xE_out[(int64_t)(r0 + q) * dm.nE1_tot + e1o + o] = mk<float>(vr[i], vi[i]);
                            else tT_out[(int64_t)(r0 + q) * dm.nT_tot + to + (o - nE)] = mk<float>(vr[i], vi[i]);
                        }
                    }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
        if (*fail) break;
        // an element without edge unknowns issued no early copy of the next element's W
        if (t == 0 && !a_pending && next < n_items) a_pending = issue_a(next);
    }
    // a copy still in flight after a failure lands before the CTA leaves (bounded)
    if (t == 0 && a_pending) mbar_wait_bounded(bar_a, ph_a);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols) : "memory");
}

static int tc_block(int R) { return R <= 16 ? 16 : (R <= 32 ? 32 : 64); }

size_t tc_smem_bytes(int maxE1, int maxT, int R, int* a_bytes) {
    const int Kp = round8(std::max(1, maxE1));
    // the MMA reads 16 row groups of each plane: the imaginary plane's view may extend
    // 16 row groups past its start, so the buffer holds 2 x 16 row groups
    (void)maxT;
    const size_t plane = (size_t)16 * (Kp / 4) * 128;
    const size_t a = 2 * plane;
    const size_t b = 2 * (size_t)(tc_block(R) / 8) * (Kp / 4) * 128;
    if (a_bytes) *a_bytes = (int)a;
    return 1024 + a + b;
}

template <int NB>
static void tc_launch_t(const DevModel& dm, const float* W, const int64_t* w_off, const int* items, int n_items,
                        const double2* z, double zsign, void* xE, void* tT, int R, const int* done, cudaStream_t st,
                        int maxT) {
    int a_bytes = 0;
    const size_t sm = tc_smem_bytes(dm.maxE1, maxT, R, &a_bytes);
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pass1_tc<NB>, 128, sm);
    // tensor memory: 512 columns per SM shared by the resident CTAs
    const int cols = NB * 2 < 32 ? 32 : NB * 2;
    per = std::max(1, std::min(per, 512 / cols));
    const int grid = std::max(1, std::min(n_items, per * std::max(1, nsm)));
    k_pass1_tc<NB><<<grid, 128, sm, st>>>(dm, W, w_off, items, n_items, z, zsign, R, (cpx<float>*)xE, (cpx<float>*)tT,
                                          done, a_bytes);
}

void launch_pass1_tc(const DevModel& dm, const float* W, const int64_t* w_off, const int* items, int n_items,
                     const double2* z, double zsign, void* xE, void* tT, int R, const int* done, cudaStream_t st, int maxT) {
    switch (tc_block(R)) {
        case 16: tc_launch_t<16>(dm, W, w_off, items, n_items, z, zsign, xE, tT, R, done, st, maxT); break;
        case 32: tc_launch_t<32>(dm, W, w_off, items, n_items, z, zsign, xE, tT, R, done, st, maxT); break;
        default: tc_launch_t<64>(dm, W, w_off, items, n_items, z, zsign, xE, tT, R, done, st, maxT);
    }
}

void set_tc_limits(int maxE1, int maxT) {
    for (int R : {16, 32, 64}) {
        const int b = (int)tc_smem_bytes(maxE1, maxT, R, nullptr);
        if (R == 16) cudaFuncSetAttribute(k_pass1_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (R == 32) cudaFuncSetAttribute(k_pass1_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (R == 64) cudaFuncSetAttribute(k_pass1_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
}

}  // namespace ddh
