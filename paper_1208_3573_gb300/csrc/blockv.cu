// Block-diagonal V (DIAF_RULE_BLOCK): the apply's V^-1 as one dense LU with
// partial pivoting per diagonal block (at most kBlockMax rows), factored once
// when the apply is prepared; every apply then solves all blocks at once,
// one warp per block.
#include "plan.cuh"
#include "sparse.cuh"

namespace {

constexpr int kBlockMax = 64;

// starts[i] = 1 where a block begins; a decreasing block id marks bad input
__global__ void block_flags_kernel(int n, const int32_t* __restrict__ blk, int32_t* __restrict__ flag,
                                   uint32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool start = i == 0 || blk[i] != blk[i - 1];
  if (i > 0 && blk[i] < blk[i - 1]) atomicOr(status, DEV_ST_BAD_INPUT);
  flag[i] = start ? 1 : 0;
}

__global__ void block_starts_kernel(int n, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                    int32_t* __restrict__ bstart, const int32_t* __restrict__ nb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) bstart[pos[i]] = i;
  if (i == 0) bstart[*nb] = n;
}

template <class S>
__device__ __forceinline__ double mag2(S v) { return (double)sc_abs2(v); }

// One CTA of kBlockMax threads per block: the dense block of V (column-major,
// leading dimension kBlockMax) from V's CSC, then LU with partial pivoting
// (pivot: the largest modulus, the lower row on ties).  Output: blu (column c
// of the block at (start + c) * kBlockMax), bpiv (block-local pivot row).
template <class S>
__global__ void __launch_bounds__(kBlockMax)
    block_lu_kernel(const int32_t* __restrict__ bstart, const int32_t* __restrict__ Vcp,
                    const int32_t* __restrict__ Vri, const S* __restrict__ Vv, S* __restrict__ blu,
                    int32_t* __restrict__ bpiv, uint32_t* status) {
  extern __shared__ __align__(16) unsigned char blu_smem[];
  S* M = reinterpret_cast<S*>(blu_smem);  // kBlockMax x kBlockMax
  __shared__ double pm[kBlockMax];
  __shared__ int pr[kBlockMax];
  const int b = blockIdx.x, t = threadIdx.x;
  const int s0 = bstart[b], nb = bstart[b + 1] - s0;
  if (nb > kBlockMax) {
    if (t == 0) atomicOr(status, DEV_ST_CAPACITY);
    return;
  }
  for (int i = t; i < kBlockMax * kBlockMax; i += kBlockMax) M[i] = sc_zero<S>();
  __syncthreads();
  if (t < nb) {
    const int j = s0 + t;
    for (int p = Vcp[j]; p < Vcp[j + 1]; ++p) {
      const int r = Vri[p] - s0;
      if (r < 0 || r >= nb) {
        atomicOr(status, DEV_ST_BAD_INPUT);  // an entry outside the diagonal block
        continue;
      }
      M[r + t * kBlockMax] = Vv[p];
    }
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    pm[t] = (t >= c && t < nb) ? mag2(M[t + c * kBlockMax]) : -1.0;
    pr[t] = t;
    __syncthreads();
    for (int o = kBlockMax / 2; o > 0; o >>= 1) {  // argmax, lower row on ties
      if (t < o) {
        const double a = pm[t], bb = pm[t + o];
        if (bb > a || (bb == a && pr[t + o] < pr[t])) { pm[t] = bb; pr[t] = pr[t + o]; }
      }
      __syncthreads();
    }
    const int p = pr[0];
    const bool zero = !(pm[0] > 0.0);
    __syncthreads();
    if (zero) {
      if (t == 0) {
        atomicOr(status, DEV_ST_SINGULAR);
        bpiv[s0 + c] = c;
      }
      continue;
    }
    if (p != c && t < nb) {  // swap rows c and p (thread t: column t)
      const S x = M[c + t * kBlockMax];
      M[c + t * kBlockMax] = M[p + t * kBlockMax];
      M[p + t * kBlockMax] = x;
    }
    if (t == 0) bpiv[s0 + c] = p;
    __syncthreads();
    const S d = M[c + c * kBlockMax];
    if (t > c && t < nb) M[t + c * kBlockMax] = M[t + c * kBlockMax] * ((1.0 / sc_abs2(d)) * sc_conj(d));
    __syncthreads();
    if (t > c && t < nb) {
      const S l = M[t + c * kBlockMax];
      for (int q = c + 1; q < nb; ++q) M[t + q * kBlockMax] -= l * M[c + q * kBlockMax];
    }
    __syncthreads();
  }
  for (int q = 0; q < nb; ++q) blu[(size_t)(s0 + q) * kBlockMax + t] = M[t + q * kBlockMax];
}

// t_b = U^-1 L^-1 P x_b for every block, one warp per block, the block's
// vector in shared memory
template <class S>
__global__ void block_solve_kernel(int nblocks, const int32_t* __restrict__ bstart, const S* __restrict__ blu,
                                   const int32_t* __restrict__ bpiv, const S* __restrict__ x, S* __restrict__ tout) {
  constexpr int kW = 4;  // warps per CTA
  __shared__ S y[kW][kBlockMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * kW + w;
  if (b >= nblocks) return;
  const int s0 = bstart[b], nb = bstart[b + 1] - s0;
  for (int r = lane; r < nb; r += 32) y[w][r] = x[s0 + r];
  __syncwarp();
  if (lane == 0)
    for (int c = 0; c < nb; ++c) {
      const int p = bpiv[s0 + c];
      if (p != c) { const S v = y[w][c]; y[w][c] = y[w][p]; y[w][p] = v; }
    }
  __syncwarp();
  for (int c = 0; c < nb; ++c) {  // L (unit lower)
    const S yc = y[w][c];
    const S* col = blu + (size_t)(s0 + c) * kBlockMax;
    for (int r = c + 1 + lane; r < nb; r += 32) y[w][r] -= col[r] * yc;
    __syncwarp();
  }
  for (int c = nb - 1; c >= 0; --c) {  // U
    const S* col = blu + (size_t)(s0 + c) * kBlockMax;
    const S d = col[c];
    const S yc = y[w][c] * ((1.0 / sc_abs2(d)) * sc_conj(d));
    __syncwarp();
    if (lane == 0) y[w][c] = yc;
    for (int r = lane; r < c; r += 32) y[w][r] -= col[r] * yc;
    __syncwarp();
  }
  for (int r = lane; r < nb; r += 32) tout[s0 + r] = y[w][r];
}

template <class S>
cudaError_t block_prepare_t(int n, const int32_t* blk, const int32_t* Vcp, const int32_t* Vri, const S* Vv,
                            BlockLu& B, int32_t* work, uint32_t* status, cudaStream_t s) {
  int32_t* flag = work;
  int32_t* pos = work + n;
  int32_t* bs = work + 2 * n;  // scan block sums
  block_flags_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, blk, flag, status);
  DIAF_COUNT_LAUNCH();
  exclusive_scan_i32(flag, pos, n, bs, s);
  // number of blocks = pos[n-1] + flag[n-1]
  int32_t last[2] = {0, 0};
  cudaMemcpyAsync(&last[0], pos + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&last[1], flag + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  B.nblocks = last[0] + last[1];
  int32_t* nbdev = bs;  // reuse: the block count on the device
  cudaMemcpyAsync(nbdev, &B.nblocks, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  block_starts_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, flag, pos, B.bstart, nbdev);
  DIAF_COUNT_LAUNCH();
  const size_t smem = sizeof(S) * kBlockMax * kBlockMax;
  static int configured_device = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    e = cudaFuncSetAttribute(block_lu_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  block_lu_kernel<S><<<B.nblocks, kBlockMax, smem, s>>>(B.bstart, Vcp, Vri, Vv, (S*)B.lu, B.piv, status);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}

}  // namespace

size_t block_lu_elems(int n) { return (size_t)n * kBlockMax; }

cudaError_t block_prepare(int n, bool cplx, const int32_t* blk, const int32_t* Vcp, const int32_t* Vri,
                          const void* Vv, BlockLu& B, int32_t* work, uint32_t* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return cplx ? block_prepare_t<Cx<double>>(n, blk, Vcp, Vri, (const Cx<double>*)Vv, B, work, status, s)
              : block_prepare_t<double>(n, blk, Vcp, Vri, (const double*)Vv, B, work, status, s);
}

cudaError_t block_solve(const BlockLu& B, bool cplx, const void* x, void* t, cudaStream_t s) {
  if (B.nblocks <= 0) return cudaSuccess;
  const int grid = ceil_div(B.nblocks, 4);
  if (cplx)
    block_solve_kernel<Cx<double>><<<grid, 128, 0, s>>>(B.nblocks, B.bstart, (const Cx<double>*)B.lu, B.piv,
                                                        (const Cx<double>*)x, (Cx<double>*)t);
  else
    block_solve_kernel<double><<<grid, 128, 0, s>>>(B.nblocks, B.bstart, (const double*)B.lu, B.piv,
                                                    (const double*)x, (double*)t);
  DIAF_COUNT_LAUNCH();
  return cudaGetLastError();
}
