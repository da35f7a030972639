// etd_ensemble.cuh -- one persistent launch per time step of a batched
// ensemble (independent problems of uneven size, Section 7's scheme on each).
//
// A step of one instance is its dim line sweeps in axis order (FIRST, [MIDDLE],
// LAST); sweep a of instance i may start only when every block of sweep a-1 of
// instance i has finished.  The step of the whole ensemble is one work list of
// (axis, instance, block) items, ordered on the host so that every item's
// dependencies come earlier in the list.  A grid of resident blocks takes items
// in list order from a device counter; a block whose item depends on sweep a-1
// of its instance waits, with a bounded wait, for that sweep's completion
// counter.  Every item it waits for was taken earlier by a running block that
// waits only on items earlier still, so the waits always end (and a wait that
// does not end within the limit records where and gives up: ETD_ERR_TIMEOUT).
// The last block to leave the loop resets the counters for the next launch.
#pragma once

#include "etd_sweep.cuh"

namespace etd {

__device__ __forceinline__ unsigned long long ens_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ens_ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 only.  Waits until *ctr >= need; false if the ensemble's status is
// already set (another wait gave up) or this wait exceeds its limit (then the
// status records instance and axis).  Two limits: %globaltimer and a poll count.
__device__ __forceinline__ bool ens_wait(const int *ctr, int need, int *status, long long wait_ns, int inst,
                                         int axis) {
  const unsigned long long t0 = ens_globaltimer();
  for (unsigned it = 0; it < (1u << 24); ++it) {
    if (ens_ld_acquire(ctr) >= need) return true;
    if (*(volatile int *)status != 0) return false;
    if ((it & 15) == 15 && (long long)(ens_globaltimer() - t0) > wait_ns) break;
    __nanosleep(128);
  }
  if (atomicCAS(status, 0, 1) == 0) {
    status[1] = inst;
    status[2] = axis;
  }
  return false;
}

// one sweep's item, compiled as its own function so that the register
// allocation of each sweep kind is that of its own kernel (TAG: one copy per
// kernel; ptxas 13.0 fails on a non-inlined function shared by two kernels)
// (the dynamic shared memory is named here, not passed in, so that its
// accesses stay shared-memory instructions rather than generic ones)
// The item's arguments are copied to shared memory first: the sweep reads
// dozens of their fields (table pointers, coefficients), which would otherwise
// be global loads on the critical path.
template <typename R, int S, int L, bool CONTIG, int KIND, int TAG, bool CIRCF>
__device__ __noinline__ void ens_sweep(const SweepArgs<R> *A, int b, double t_eval, R exp_mt) {
  extern __shared__ __align__(16) unsigned char ens_smem[];
  static_assert(sizeof(SweepArgs<R>) % 8 == 0, "arguments copied in 8-byte pieces");
  __shared__ __align__(16) int2 s_args[sizeof(SweepArgs<R>) / 8];
  const int2 *src = reinterpret_cast<const int2 *>(A);
  for (int i = threadIdx.x; i < (int)(sizeof(SweepArgs<R>) / 8); i += blockDim.x) s_args[i] = src[i];
  __syncthreads();
  sweep_block<R, S, L, CONTIG, KIND, 1, false, true, CIRCF>(*reinterpret_cast<const SweepArgs<R> *>(s_args), b,
                                                            ens_smem, t_eval, exp_mt);
  __syncthreads();  // every thread is done with the arguments before the next item's copy
}

// one work item of axis a with chunk lengths L0 (axis 0) and LS (axes 1, 2)
template <typename R, int S, int L0, int LS, int DIM>
__device__ __forceinline__ void ens_item(const EnsArgs<R> &E, int a, int inst, int b) {
  constexpr int TAG = L0 * 100 + LS;
  const SweepArgs<R> *A = E.args[a] + inst;
  const bool circ = A->circ_fwd != 0;  // periodic whole-chunk lines: circulant sweep
  if (a == 0) {
    if (circ) ens_sweep<R, S, L0, true, SWEEP_FIRST, TAG, true>(A, b, E.t_eval[0], E.exp_mt[0]);
    else ens_sweep<R, S, L0, true, SWEEP_FIRST, TAG, false>(A, b, E.t_eval[0], E.exp_mt[0]);
  } else if (DIM == 3 && a == 1) {
    if (circ) ens_sweep<R, S, LS, false, SWEEP_MIDDLE, TAG, true>(A, b, E.t_eval[1], E.exp_mt[1]);
    else ens_sweep<R, S, LS, false, SWEEP_MIDDLE, TAG, false>(A, b, E.t_eval[1], E.exp_mt[1]);
  } else {
    if (circ) ens_sweep<R, S, LS, false, SWEEP_LAST, TAG, true>(A, b, E.t_eval[DIM - 1], E.exp_mt[DIM - 1]);
    else ens_sweep<R, S, LS, false, SWEEP_LAST, TAG, false>(A, b, E.t_eval[DIM - 1], E.exp_mt[DIM - 1]);
  }
}

template <typename R, int S, int L0, int LS, int DIM>
__global__ void __launch_bounds__(ETD_MAX_THREADS) ensemble_step_kernel(const __grid_constant__ EnsArgs<R> E) {
  __shared__ int s_item, s_next, s_go;
  const int tid = threadIdx.x;
  if (tid == 0) s_item = (int)atomicAdd(E.queue, 1u);
  __syncthreads();
  int it = s_item;
  while (it < E.nitems) {
    const int2 w = E.items[it];
    const int a = w.x >> 24, inst = w.x & 0xffffff, b = w.y;
    if (tid == 0) {
      // take the next item now: the atomic's latency overlaps this item.  The
      // smallest unfinished item is always running (every item it depends on
      // is smaller), so holding one item ahead cannot stall the list.
      s_next = (int)atomicAdd(E.queue, 1u);
      bool go = true;
      if (a > 0)
        go = ens_wait(E.done + (size_t)(a - 1) * E.ninst + inst, E.args[a - 1][inst].nblocks, E.status,
                      E.wait_ns, inst, a);
      else
        go = *(volatile int *)E.status == 0;
      if (go) __threadfence();  // the waited-for sweep's stores are visible to the whole block
      s_go = go;
    }
    __syncthreads();
    const int next = s_next;
    const bool go = s_go;
    if (go) ens_item<R, S, L0, LS, DIM>(E, a, inst, b);
    __syncthreads();  // every thread's stores of this item are issued; smem free for the next item
    if (tid == 0 && go && a < DIM - 1) {
      __threadfence();
      atomicAdd(E.done + (size_t)a * E.ninst + inst, 1);
    }
    it = next;
  }
  // the last block out resets the counters for the next launch (stream order)
  __shared__ int s_last;
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(E.queue + 1, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int i = tid; i < (DIM - 1) * E.ninst; i += blockDim.x) E.done[i] = 0;
    if (tid == 0) {
      E.queue[0] = 0;
      E.queue[1] = 0;
    }
  }
}

// Host side.  resident != nullptr: only report the resident blocks of this
// configuration (blocks per SM x SMs); otherwise launch `grid` blocks on s.
template <typename R, int S, int L0, int LS, int DIM>
cudaError_t ensemble_one(const EnsArgs<R> &E, int nthreads, size_t smem, int grid, cudaStream_t s, int *resident) {
  auto fn = ensemble_step_kernel<R, S, L0, LS, DIM>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (resident) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nthreads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    *resident = (e == cudaSuccess) ? per_sm * nsm : 0;
    return e;
  }
  if (grid < 1) return cudaErrorInvalidConfiguration;
  fn<<<grid, nthreads, smem, s>>>(E);
  return cudaGetLastError();
}

// dispatch over species and chunk lengths for one element type and dim
template <typename R, int DIM>
cudaError_t ensemble_any(const EnsArgs<R> &E, int nspecies, int L0, int LS, int nthreads, size_t smem, int grid,
                         cudaStream_t s, int *resident) {
  constexpr int LA = sizeof(R) == 4 ? 8 : 4, LB = sizeof(R) == 4 ? 16 : 8;
  const int key = nspecies * 100 + (L0 == LB) * 10 + (LS == LB);
  if ((L0 != LA && L0 != LB) || (LS != LA && LS != LB)) return cudaErrorInvalidValue;
  switch (key) {
    case 100: return ensemble_one<R, 1, LA, LA, DIM>(E, nthreads, smem, grid, s, resident);
    case 101: return ensemble_one<R, 1, LA, LB, DIM>(E, nthreads, smem, grid, s, resident);
    case 110: return ensemble_one<R, 1, LB, LA, DIM>(E, nthreads, smem, grid, s, resident);
    case 111: return ensemble_one<R, 1, LB, LB, DIM>(E, nthreads, smem, grid, s, resident);
    case 200: return ensemble_one<R, 2, LA, LA, DIM>(E, nthreads, smem, grid, s, resident);
    case 201: return ensemble_one<R, 2, LA, LB, DIM>(E, nthreads, smem, grid, s, resident);
    case 210: return ensemble_one<R, 2, LB, LA, DIM>(E, nthreads, smem, grid, s, resident);
    case 211: return ensemble_one<R, 2, LB, LB, DIM>(E, nthreads, smem, grid, s, resident);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace etd
