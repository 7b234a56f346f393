// Device twins of the seeded count samplers in synth/counts.py.
//
// Same Philox4x32-10 definition (Salmon et al., SC'11), same counters, same
// integer thresholds, so the counts are bit-identical to the CPU samplers.
// One CTA per basis (grid-stride): a shared-memory histogram of that basis'
// shots, then one coalesced write of its 2^n counts.  Input synthesis only:
// nothing here is part of the estimator.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

constexpr uint32_t STREAM_CDF = 0x11, STREAM_GHZ = 0x22, STREAM_PROD = 0x33, STREAM_SPLIT = 0x44;

template <typename OutT>
__device__ void write_row(const int32_t *h, OutT *row, int d) {
  for (int o = threadIdx.x; o < d; o += blockDim.x) row[o] = (OutT)h[o];
}

// Set bits among the first c bits of node `node`'s word stream for basis b,
// calls g = g0, g0 + step, ... (Binomial(c, 1/2) summed over the caller's
// share of the calls).
__device__ __forceinline__ int32_t fair_bits(int32_t c, uint32_t b, uint32_t node, uint32_t k0, uint32_t k1,
                                             int32_t g0, int32_t step) {
  int32_t acc = 0;
  const int32_t calls = (c + 127) >> 7;
  for (int32_t g = g0; g < calls; g += step) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)g, b, STREAM_SPLIT, node), k0, k1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int32_t nb = min(max(c - (g * 128 + 32 * k), 0), 32);
      const uint32_t mask = nb >= 32 ? 0xFFFFFFFFu : ((1u << nb) - 1u);
      acc += __popc(ws[k] & mask);
    }
  }
  return acc;
}

// Maximally mixed state by binary splitting of each basis' shots (qubit 1
// first); node (q, v) lives in slot v << (n - q) of the shared array, which
// its left child keeps: c0 = Binomial(c, 1/2) stays, c - c0 moves half a
// subtree to the right.  Warps share a node's calls at the first six levels,
// threads own whole nodes below.
template <typename OutT>
__global__ void gen_mixed_kernel(int n, int64_t b0, int64_t nb, int64_t shots, uint32_t k0, uint32_t k1,
                                 OutT *__restrict__ counts) {
  extern __shared__ int32_t h[];
  const int d = 1 << n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int64_t j = blockIdx.x; j < nb; j += gridDim.x) {
    const uint32_t b = (uint32_t)(b0 + j);
    for (int o = threadIdx.x; o < d; o += blockDim.x) h[o] = 0;
    __syncthreads();
    if (threadIdx.x == 0) h[0] = (int32_t)shots;
    __syncthreads();
    for (int q = 0; q < n; ++q) {
      const int half = 1 << (n - q - 1);
      if (q < 6) {
        for (int v = warp; v < (1 << q); v += nwarps) {
          const int slot = v << (n - q);
          const int32_t c = h[slot];
          int32_t c0 = fair_bits(c, b, (1u << q) | (uint32_t)v, k0, k1, lane, 32);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) c0 += __shfl_xor_sync(0xffffffffu, c0, o);
          __syncwarp();
          if (lane == 0) {
            h[slot] = c0;
            h[slot + half] = c - c0;
          }
        }
      } else {
        for (int v = threadIdx.x; v < (1 << q); v += blockDim.x) {
          const int slot = v << (n - q);
          const int32_t c = h[slot];
          const int32_t c0 = fair_bits(c, b, (1u << q) | (uint32_t)v, k0, k1, 0, 1);
          h[slot] = c0;
          h[slot + half] = c - c0;
        }
      }
      __syncthreads();
    }
    write_row(h, counts + j * (int64_t)d, d);
    __syncthreads();
  }
}

template <typename OutT>
__global__ void gen_cdf_kernel(const uint32_t *__restrict__ thr, int n, int64_t b0, int64_t nb,
                               int64_t shots, uint32_t k0, uint32_t k1, OutT *__restrict__ counts) {
  extern __shared__ int32_t h[];
  const int d = 1 << n;
  for (int64_t j = blockIdx.x; j < nb; j += gridDim.x) {
    const int64_t b = b0 + j;
    for (int o = threadIdx.x; o < d; o += blockDim.x) h[o] = 0;
    __syncthreads();
    const uint32_t *t = thr + b * (int64_t)(d - 1);
    for (int64_t g = threadIdx.x; g * 4 < shots; g += blockDim.x) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)b, STREAM_CDF, 0u), k0, k1);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
      for (int q = 0; q < 4 && g * 4 + q < shots; ++q) {
        const uint32_t u = ws[q];
        int lo = 0, hi = d - 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (t[mid] <= u) lo = mid + 1;
          else hi = mid;
        }
        atomicAdd(&h[lo], 1);
      }
    }
    __syncthreads();
    write_row(h, counts + j * (int64_t)d, d);
    __syncthreads();
  }
}

template <typename OutT>
__global__ void gen_ghz_kernel(int n, uint32_t noise_thr, int64_t b0, int64_t nb, int64_t shots,
                               uint32_t k0, uint32_t k1, OutT *__restrict__ counts) {
  extern __shared__ int32_t h[];
  const int d = 1 << n;
  for (int64_t j = blockIdx.x; j < nb; j += gridDim.x) {
    const int64_t b = b0 + j;
    uint32_t zmask = 0;
    int ny = 0;
    int64_t x = b;
    for (int q = 0; q < n; ++q) {  // q-th least significant qubit
      const int a = (int)(x % 3);
      x /= 3;
      if (a == 2) zmask |= 1u << q;
      if (a == 1) ++ny;
    }
    const uint32_t par = (uint32_t)((ny >> 1) & 1);
    for (int o = threadIdx.x; o < d; o += blockDim.x) h[o] = 0;
    __syncthreads();
    for (int64_t s = threadIdx.x; s < shots; s += blockDim.x) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)b, STREAM_GHZ, 0u), k0, k1);
      const uint32_t u = w.y & (uint32_t)(d - 1);
      uint32_t o;
      if (w.x < noise_thr) o = u;
      else if (zmask) o = (u & ~zmask) | ((w.z & 1u) ? zmask : 0u);
      else if (ny & 1) o = u;
      else o = ((uint32_t)(__popc(u) & 1) != par) ? (u ^ 1u) : u;
      atomicAdd(&h[o], 1);
    }
    __syncthreads();
    write_row(h, counts + j * (int64_t)d, d);
    __syncthreads();
  }
}

// Shot records of the same GHZ sampler: rec[j][s] = outcome of shot s of basis b0 + j.
__global__ void gen_ghz_records_kernel(int n, uint32_t noise_thr, int64_t b0, int64_t nb, int64_t shots,
                                       uint32_t k0, uint32_t k1, uint16_t *__restrict__ rec) {
  const int d = 1 << n;
  const int64_t total = nb * shots;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / shots, s = e - j * shots;
    const int64_t b = b0 + j;
    uint32_t zmask = 0;
    int ny = 0;
    int64_t x = b;
    for (int q = 0; q < n; ++q) {
      const int a = (int)(x % 3);
      x /= 3;
      if (a == 2) zmask |= 1u << q;
      if (a == 1) ++ny;
    }
    const uint32_t par = (uint32_t)((ny >> 1) & 1);
    const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)b, STREAM_GHZ, 0u), k0, k1);
    const uint32_t u = w.y & (uint32_t)(d - 1);
    uint32_t o;
    if (w.x < noise_thr) o = u;
    else if (zmask) o = (u & ~zmask) | ((w.z & 1u) ? zmask : 0u);
    else if (ny & 1) o = u;
    else o = ((uint32_t)(__popc(u) & 1) != par) ? (u ^ 1u) : u;
    rec[e] = (uint16_t)o;
  }
}

template <typename OutT>
__global__ void gen_product_kernel(const uint32_t *__restrict__ thr, int n, int64_t b0, int64_t nb,
                                   int64_t shots, uint32_t k0, uint32_t k1, OutT *__restrict__ counts) {
  extern __shared__ int32_t h[];
  __shared__ uint32_t tq[32];
  const int d = 1 << n;
  for (int64_t j = blockIdx.x; j < nb; j += gridDim.x) {
    const int64_t b = b0 + j;
    if (threadIdx.x == 0) {
      int64_t x = b;
      for (int q = n - 1; q >= 0; --q) {  // q: qubit index from the most significant
        const int a = (int)(x % 3);
        x /= 3;
        tq[q] = thr[q * 3 + a];
      }
    }
    for (int o = threadIdx.x; o < d; o += blockDim.x) h[o] = 0;
    __syncthreads();
    for (int64_t s = threadIdx.x; s < shots; s += blockDim.x) {
      uint32_t o = 0;
      for (int call = 0; call * 4 < n; ++call) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)b, STREAM_PROD, (uint32_t)call), k0, k1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        for (int jj = 0; jj < 4; ++jj) {
          const int q = call * 4 + jj;
          if (q >= n) break;
          if (ws[jj] >= tq[q]) o |= 1u << (n - 1 - q);
        }
      }
      atomicAdd(&h[o], 1);
    }
    __syncthreads();
    write_row(h, counts + j * (int64_t)d, d);
    __syncthreads();
  }
}

template <typename K>
int launch_cfg(K kern, int n, int64_t nb, int &grid) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = (int)(sizeof(int32_t) << n);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  grid = sms * 3;
  if (grid > nb) grid = (int)nb;
  return smem;
}

}  // namespace

extern "C" {

// kind: 0 int32 counts, 1 int16 counts.  Returns a cudaError_t code.
int synth_gen_cdf(const uint32_t *thr, int n, int64_t b0, int64_t nb, int64_t shots, uint64_t seed,
                  void *counts, int kind, cudaStream_t s) {
  int grid;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (kind == 1) {
    int smem = launch_cfg(gen_cdf_kernel<int16_t>, n, nb, grid);
    gen_cdf_kernel<int16_t><<<grid, 256, smem, s>>>(thr, n, b0, nb, shots, k0, k1, (int16_t *)counts);
  } else {
    int smem = launch_cfg(gen_cdf_kernel<int32_t>, n, nb, grid);
    gen_cdf_kernel<int32_t><<<grid, 256, smem, s>>>(thr, n, b0, nb, shots, k0, k1, (int32_t *)counts);
  }
  return (int)cudaGetLastError();
}

int synth_gen_ghz(int n, uint32_t noise_thr, int64_t b0, int64_t nb, int64_t shots, uint64_t seed,
                  void *counts, int kind, cudaStream_t s) {
  int grid;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (kind == 1) {
    int smem = launch_cfg(gen_ghz_kernel<int16_t>, n, nb, grid);
    gen_ghz_kernel<int16_t><<<grid, 512, smem, s>>>(n, noise_thr, b0, nb, shots, k0, k1, (int16_t *)counts);
  } else {
    int smem = launch_cfg(gen_ghz_kernel<int32_t>, n, nb, grid);
    gen_ghz_kernel<int32_t><<<grid, 512, smem, s>>>(n, noise_thr, b0, nb, shots, k0, k1, (int32_t *)counts);
  }
  return (int)cudaGetLastError();
}

int synth_gen_product(const uint32_t *thr, int n, int64_t b0, int64_t nb, int64_t shots, uint64_t seed,
                      void *counts, int kind, cudaStream_t s) {
  int grid;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (kind == 1) {
    int smem = launch_cfg(gen_product_kernel<int16_t>, n, nb, grid);
    gen_product_kernel<int16_t><<<grid, 512, smem, s>>>(thr, n, b0, nb, shots, k0, k1, (int16_t *)counts);
  } else {
    int smem = launch_cfg(gen_product_kernel<int32_t>, n, nb, grid);
    gen_product_kernel<int32_t><<<grid, 512, smem, s>>>(thr, n, b0, nb, shots, k0, k1, (int32_t *)counts);
  }
  return (int)cudaGetLastError();
}

int synth_gen_mixed(int n, int64_t b0, int64_t nb, int64_t shots, uint64_t seed, void *counts, int kind,
                    cudaStream_t s) {
  int grid;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (kind == 1) {
    int smem = launch_cfg(gen_mixed_kernel<int16_t>, n, nb, grid);
    gen_mixed_kernel<int16_t><<<grid, 256, smem, s>>>(n, b0, nb, shots, k0, k1, (int16_t *)counts);
  } else {
    int smem = launch_cfg(gen_mixed_kernel<int32_t>, n, nb, grid);
    gen_mixed_kernel<int32_t><<<grid, 256, smem, s>>>(n, b0, nb, shots, k0, k1, (int32_t *)counts);
  }
  return (int)cudaGetLastError();
}

int synth_gen_ghz_records(int n, uint32_t noise_thr, int64_t b0, int64_t nb, int64_t shots,
                          uint64_t seed, uint16_t *rec, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  gen_ghz_records_kernel<<<sms * 8, 256, 0, s>>>(n, noise_thr, b0, nb, shots, (uint32_t)seed,
                                                (uint32_t)(seed >> 32), rec);
  return (int)cudaGetLastError();
}

}  // extern "C"
