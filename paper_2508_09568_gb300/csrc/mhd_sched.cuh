// Device-side scheduler of asynchronous per-patch time stepping (mhd_bunch_advance_async).
//
// Every round of the asynchronous advance (DISPATCH's patches at their own times, Sec. 2.2,
// updated in bunches of ready patches, Sec. 2.4) is a sequence of stream-ordered launches
// with no host round trip:
//   async_commit_kernel    the previous round's patches: t_old <- t_cur, t_cur <- t_cur + dt
//                          (t_span for a patch that arrived), slice flipped;
//   async_ready_kernel     a flag per patch: short of t_span and no neighbour (an owner of
//                          a cell of its guard zone) at an earlier time;
//   async_list_kernel      the flagged patches in ascending order and their tiles (one CTA,
//                          block-wide scans);
//   fill_interp_kernel     guard zones of the listed patches at their own times;
//   cfl_patch_kernel       each listed patch's maximum CFL rate;
//   async_clamp_kernel     dt = courant / rate, clipped to what is left of t_span, recorded;
//   step_kernel (ASYNC)    the update of the listed tiles, each patch by its own dt.
// The host enqueues rounds in batches and reads each batch's record afterwards.  The
// readiness test reads t_cur after the commit, as a host scheduler would between rounds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mhd_common.cuh"

namespace mhd {

constexpr int kSchedThreads = 1024;   // async_list_kernel: one CTA of 32 warps

// Exclusive scan of v over the 1024 threads of the block; *total receives the sum.
// ws: 32 ints of shared memory, free again on return.
__device__ __forceinline__ int block_exscan(int v, int* ws, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const int prefix = (wid ? ws[wid - 1] : 0) + x - v;
    *total = ws[31];
    __syncthreads();
    return prefix;
}

__global__ void async_commit_kernel(const int* __restrict__ list, const int* n_ptr, const double* __restrict__ dt,
                                    const unsigned char* __restrict__ last, double t_span, double* t_old,
                                    double* t_cur, int* slice) {
    const int n = *n_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = list[i];
        const double t = t_cur[p];
        t_old[p] = t;
        t_cur[p] = last[i] ? t_span : t + dt[i];
        slice[p] ^= 1;
    }
}

// ready[p] = 1 when patch p is short of t_span and no neighbour is at an earlier time
// (nothing is ready once a round has failed: *abort != 0)
__global__ void async_ready_kernel(int npatch, const int* __restrict__ nb_off, const int* __restrict__ nb_idx,
                                   const double* __restrict__ t_cur, double t_span, const unsigned* abort,
                                   int* ready) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npatch) return;
    const double tp = t_cur[p];
    int ok = (*abort == 0u) && tp < t_span;
    const int k1 = nb_off[p + 1];
#pragma unroll 4
    for (int k = nb_off[p]; k < k1; ++k) ok &= t_cur[nb_idx[k]] >= tp;   // all loads independent
    ready[p] = ok;
}

// The ready patches in ascending order (list, *n_out), their tiles patch by patch in the
// natural tile order (tiles, *ntiles_out), and their rate maxima zeroed.  One CTA.
__global__ void __launch_bounds__(kSchedThreads) async_list_kernel(int npatch, const int* __restrict__ ready,
                                                                   const int* __restrict__ tfirst,
                                                                   const int* __restrict__ tcount,
                                                                   const int4* __restrict__ tnat, int* list,
                                                                   int* n_out, int4* tiles, int* ntiles_out,
                                                                   unsigned long long* rate_max) {
    __shared__ int ws[32];
    int count = 0, tcnt = 0;
    for (int base = 0; base < npatch; base += blockDim.x) {
        const int p = base + threadIdx.x;
        const int r = p < npatch ? ready[p] : 0;
        int tot = 0, ttot = 0;
        const int pos = block_exscan(r, ws, &tot);
        const int nt = r ? tcount[p] : 0;
        const int tpos = block_exscan(nt, ws, &ttot);
        if (r) {
            list[count + pos] = p;
            rate_max[p] = 0ull;
            const int f = tfirst[p];
            for (int j = 0; j < nt; ++j) tiles[tcnt + tpos + j] = tnat[f + j];
        }
        count += tot;
        tcnt += ttot;
    }
    if (threadIdx.x == 0) {
        *n_out = count;
        *ntiles_out = tcnt;
    }
}

// dt of each listed patch: courant / its maximum CFL rate (rate_max, the bits of a
// non-negative double from cfl_patch_kernel), clipped to what is left of t_span (last = 1
// when clipped), written to dtp for the update and recorded in the round's row.  A
// non-positive or non-finite dt sets ERR_PHYS and the abort flag (later rounds schedule
// nothing) and is replaced by 0 so that the update leaves the patch unchanged.
__global__ void async_clamp_kernel(const int* __restrict__ list, const int* n_ptr,
                                   const unsigned long long* __restrict__ rate_max, double courant,
                                   const double* __restrict__ t_cur, double t_span, double* dtp, double* dt_row,
                                   unsigned char* last_row, unsigned* abort, unsigned* err) {
    const int n = *n_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = list[i];
        double d = courant / __longlong_as_double((long long)rate_max[p]);
        const double rem = t_span - t_cur[p];
        unsigned char last = 0;
        if (!(d > 0.0) || !isfinite(d)) {
            atomicOr(abort, 1u);
            atomicOr(err, ERR_PHYS);
            d = 0.0;
        } else if (d >= rem) {
            d = rem;
            last = 1;
        }
        dtp[p] = d;
        dt_row[i] = d;
        last_row[i] = last;
    }
}

// The final slice of every patch into the buffer `to`: a patch whose current slice is 1
// (held by `from`) is copied whole (8 variables of its padded block), as 4-byte words.
__global__ void async_gather_kernel(unsigned* to, const unsigned* __restrict__ from,
                                    const PatchDev* __restrict__ patches, int npatch, const int* __restrict__ slice,
                                    int real_words) {
    for (int p = blockIdx.y; p < npatch; p += gridDim.y) {
        if (!slice[p]) continue;
        const PatchDev pt = patches[p];
        const int64_t w0 = pt.off * real_words;
        const int64_t nw = (int64_t)8 * pt.X * pt.Y * pt.Z * real_words;
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nw; k += (int64_t)gridDim.x * blockDim.x)
            to[w0 + k] = from[w0 + k];
    }
}

}  // namespace mhd
