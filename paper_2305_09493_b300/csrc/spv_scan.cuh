// spv_scan.cuh -- device-wide exclusive scans for the batch kernels whose
// counts are known only on the device: out[i] = in[0] + ... + in[i-1] and
// out[n] = the total, n read from device memory (at most a host capacity),
// in three launches (tile sums, one-block scan of the sums, tile scans).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "spv_prof.h"

namespace {

// exclusive block scan of one value per thread (blockDim.x a multiple of 32)
__device__ __forceinline__ unsigned long long block_exscan(unsigned long long v, unsigned long long *total)
{
    __shared__ unsigned long long s_w[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
    #pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = lane < nw ? s_w[lane] : 0;
        #pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < nw) s_w[lane] = t;
    }
    __syncthreads();
    const unsigned long long pre = (wid ? s_w[wid - 1] : 0) + x - v;
    if (total) *total = s_w[nw - 1];
    __syncthreads();
    return pre;
}

constexpr int SC_THREADS = 256, SC_PER = 8, SC_TILE = SC_THREADS * SC_PER;

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_sums(const T *in, const long long *n_ptr, long long cap,
                                                          unsigned long long *sums)
{
    long long n = *n_ptr;
    if (n > cap) n = cap;
    const long long tiles = (n + SC_TILE - 1) / SC_TILE;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        unsigned long long v = 0;
        const long long b = t * SC_TILE + (long long)threadIdx.x * SC_PER;
        #pragma unroll
        for (int k = 0; k < SC_PER; k++)
            if (b + k < n) v += (unsigned long long)in[b + k];
        unsigned long long total;
        block_exscan(v, &total);
        if (threadIdx.x == 0) sums[t] = total;
    }
}

// one block: exclusive scan of the tile sums in place; sums[tiles] = total
__global__ void __launch_bounds__(1024) k_scan_top(const long long *n_ptr, long long cap, unsigned long long *sums,
                                                   long long *total_out)
{
    long long n = *n_ptr;
    if (n > cap) n = cap;
    const long long tiles = (n + SC_TILE - 1) / SC_TILE;
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long base = 0; base < tiles; base += 1024) {
        const long long i = base + threadIdx.x;
        const unsigned long long v = i < tiles ? sums[i] : 0;
        unsigned long long x = v;
        #pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long t = s_w[lane];
            #pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, d);
                if (lane >= d) t += y;
            }
            s_w[lane] = t;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (i < tiles) sums[i] = carry + (wid ? s_w[wid - 1] : 0) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + s_w[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[tiles] = s_carry;
        if (total_out) *total_out = (long long)s_carry;
    }
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_out(const T *in, const long long *n_ptr, long long cap,
                                                         const unsigned long long *sums, unsigned long long *out)
{
    long long n = *n_ptr;
    if (n > cap) n = cap;
    const long long tiles = (n + SC_TILE - 1) / SC_TILE;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long b = t * SC_TILE + (long long)threadIdx.x * SC_PER;
        T v[SC_PER];
        unsigned long long s = 0;
        #pragma unroll
        for (int k = 0; k < SC_PER; k++) {
            v[k] = b + k < n ? in[b + k] : (T)0;
            s += (unsigned long long)v[k];
        }
        unsigned long long pre = sums[t] + block_exscan(s, nullptr);
        #pragma unroll
        for (int k = 0; k < SC_PER; k++) {
            if (b + k < n) out[b + k] = pre;
            pre += (unsigned long long)v[k];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[tiles];
}

// blocks for work items at threads per block: at most 16 per SM
int grid_for(long long work, int threads)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    long long b = (work + threads - 1) / threads;
    const long long cap = (long long)nsm * 16;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// exclusive scan of n (device value at n_ptr, at most cap) items
template <typename T>
void scan(const T *in, const long long *n_ptr, long long cap, unsigned long long *sums, unsigned long long *out,
          long long *total, cudaStream_t st)
{
    const int g = grid_for((cap + SC_TILE - 1) / SC_TILE * SC_THREADS, SC_THREADS);
    SPV_LAUNCH("k_scan_sums", st, k_scan_sums<T><<<g, SC_THREADS, 0, st>>>(in, n_ptr, cap, sums));
    SPV_LAUNCH("k_scan_top", st, k_scan_top<<<1, 1024, 0, st>>>(n_ptr, cap, sums, total));
    SPV_LAUNCH("k_scan_out", st, k_scan_out<T><<<g, SC_THREADS, 0, st>>>(in, n_ptr, cap, sums, out));
}

}  // namespace
