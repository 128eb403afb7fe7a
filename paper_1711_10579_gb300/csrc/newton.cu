// Launchers of the persistent Newton kernel (single solves, Newton-Krylov
// batches) and of the group kernel of served requests, the scratch array of
// pf_solve_noalloc, and the kernels' dynamic shared memory.  The kernels
// themselves are in newton.cuh, compiled per block size and precision.
#include "kernels.cuh"

namespace pf {

// Entry points of one block size and precision, defined in newton.cuh and
// instantiated by newton_2f.cu, newton_2d.cu, newton_6f.cu, newton_6d.cu.
template <int BS, typename TF>
cudaError_t launch_newton_as(bool nk, const DevSys& S, const DevWork& w, const DevOpts& o,
                             int grid, int cluster, int threads, cudaStream_t st);
template <int BS, typename TF>
cudaError_t launch_group_as(const GroupJob* desc, const GroupList& list, size_t smem, int cluster,
                            cudaStream_t st);
template <int BS, typename TF>
int max_cluster_as(bool nk, int threads);

// Scratch of pf_solve_noalloc: one fixed array in device memory, so that
// entry point allocates nothing.  Every GPU that loads this library holds it
// until the process exits; every call of that entry point shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (the first call on a device does this
// set-up) and cached.
cudaError_t noalloc_scratch(void** ptr) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return cudaSuccess;
}

size_t dynamic_smem_bytes(int bs, size_t tf, bool nk, int n, const DevOpts& o, int threads) {
  size_t b = o.y_in_smem ? (size_t)n * bs * tf : 0;
  if (nk) {
    const size_t words = (size_t)(o.m + 1) * o.m + 4 * o.m + 1;
    b += (size_t)o.S * words * tf;
    b += (size_t)(threads / 32) * kMaxJ * o.S * tf;
    b += (size_t)kMaxJ * o.S * tf;
  }
  if (o.S > 1) b += (size_t)threads * bs * tf;  // batched sweep partials
  if (o.ring) {                                  // batched factor ring
    b = (b + 15) & ~(size_t)15;
    b += (size_t)threads * (tf == 4 ? FactorPipe<float>::bytes : FactorPipe<double>::bytes);
  }
  return b;
}

cudaError_t launch_newton(int bs, bool fp32, bool nk, const DevSys& S, const DevWork& w,
                          const DevOpts& o, int grid, int cluster, int threads, cudaStream_t st) {
  if (bs == 2)
    return fp32 ? launch_newton_as<2, float>(nk, S, w, o, grid, cluster, threads, st)
                : launch_newton_as<2, double>(nk, S, w, o, grid, cluster, threads, st);
  return fp32 ? launch_newton_as<6, float>(nk, S, w, o, grid, cluster, threads, st)
              : launch_newton_as<6, double>(nk, S, w, o, grid, cluster, threads, st);
}

cudaError_t launch_newton_group(int bs, bool fp32, const GroupJob* desc, const GroupList& list,
                                size_t smem, int cluster, cudaStream_t st) {
  if (list.n <= 0 || list.n > kGroupMax || cluster < 1 || cluster > 8) return cudaErrorInvalidValue;
  if (bs == 2)
    return fp32 ? launch_group_as<2, float>(desc, list, smem, cluster, st)
                : launch_group_as<2, double>(desc, list, smem, cluster, st);
  return fp32 ? launch_group_as<6, float>(desc, list, smem, cluster, st)
              : launch_group_as<6, double>(desc, list, smem, cluster, st);
}

int max_cluster(int bs, bool fp32, bool nk, int threads) {
  if (bs == 2)
    return fp32 ? max_cluster_as<2, float>(nk, threads) : max_cluster_as<2, double>(nk, threads);
  return fp32 ? max_cluster_as<6, float>(nk, threads) : max_cluster_as<6, double>(nk, threads);
}

}  // namespace pf
