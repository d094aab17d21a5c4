// ehc_noalloc.cu -- electronic-energy reduction that allocates nothing.
//
// Some callers cannot allocate device memory when they need this number: a host
// application whose device memory pool is sized once at start-up and forbids
// later cudaMalloc, a plugin running inside another code's MD loop that may not
// touch that code's allocator, or a real-time loop that must not take the
// driver's allocation locks.  ehc_electron_energy_noalloc serves them: its
// scratch (the per-block partial sums) lives in a fixed file-scope device array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ehc_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaAtomsPerBlock = 4096;   // atoms per block (16 per thread)
constexpr int kNaMaxBlocks = 4096;       // scratch slots -> at most 16,777,216 atoms
constexpr int kNaMaxDevices = 64;

// Every GPU that loads the library holds this array (4096 x 4 doubles = 128 KB)
// until the process exits.  All calls share it.
static __device__ __align__(256) double na_scratch[kNaMaxBlocks * 4];

std::mutex na_mutex;
double *na_ptr[kNaMaxDevices] = {nullptr};

__device__ __forceinline__ double na_block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

// maximum that keeps a NaN (fmax would drop it): a NaN temperature shows as max T
__device__ __forceinline__ double na_max(double a, double b) { return (a != a) ? a : ((b != b) ? b : fmax(a, b)); }

__device__ __forceinline__ double na_block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = na_max(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = -1e300;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : -1e300;
    for (int o = 16; o > 0; o >>= 1) r = na_max(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

// per block: sum T, max T, sum of int_0^T min(gamma T', cap) dT' [J m^-3]
__global__ void na_partial(int64_t n, const double *__restrict__ T, double gamma, double cap,
                           double *__restrict__ part) {
  __shared__ double sh[32];
  const int64_t b0 = (int64_t)blockIdx.x * kNaAtomsPerBlock;
  int64_t b1 = b0 + kNaAtomsPerBlock;
  if (b1 > n) b1 = n;
  double sT = 0, mT = -1e300, sE = 0;
  for (int64_t s = b0 + threadIdx.x; s < b1; s += blockDim.x) {
    const double t = T[s];
    sT += t;
    mT = na_max(mT, t);
    if (cap > 0.0 && gamma * t > cap) {
      const double Tc = cap / gamma;
      sE += 0.5 * cap * Tc + cap * (t - Tc);
    } else {
      sE += 0.5 * gamma * t * t;
    }
  }
  const double r0 = na_block_sum(sT, sh);
  const double r1 = na_block_max(mT, sh);
  const double r2 = na_block_sum(sE, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 4 + 0] = r0;
    part[blockIdx.x * 4 + 1] = r1;
    part[blockIdx.x * 4 + 2] = r2;
    part[blockIdx.x * 4 + 3] = 0.0;
  }
}

__global__ void na_final(int nb, const double *__restrict__ part, double e_scale, double *__restrict__ out) {
  __shared__ double sh[32];
  double sT = 0, mT = -1e300, sE = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    sT += part[b * 4 + 0];
    mT = na_max(mT, part[b * 4 + 1]);
    sE += part[b * 4 + 2];
  }
  const double r0 = na_block_sum(sT, sh);
  const double r1 = na_block_max(mT, sh);
  const double r2 = na_block_sum(sE, sh);
  if (threadIdx.x == 0) {
    out[0] = r0;
    out[1] = nb > 0 ? r1 : 0.0;
    out[2] = r2 * e_scale;
  }
}

// device address of the scratch array on the current device, looked up once per
// device (cudaGetSymbolAddress must run with that device current).  The cached
// address belongs to the device's current context: after cudaDeviceReset on that
// device it is stale, so the entry point must not be used across a reset.
int scratch_ptr(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EHC_E_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return EHC_E_INVAL;
  std::lock_guard<std::mutex> lk(na_mutex);
  if (!na_ptr[dev]) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, na_scratch) != cudaSuccess || !p) return EHC_E_CUDA;
    na_ptr[dev] = p;
  }
  *out = na_ptr[dev];
  return EHC_OK;
}

}  // namespace

extern "C" int ehc_electron_energy_noalloc(const double *Te_dev, int64_t n, double gamma_Ce, double Ce_cap_kB,
                                           double vatom_A3, double *out_dev, void *stream) {
  if (n < 0 || !out_dev || (n > 0 && !Te_dev) || !(gamma_Ce > 0) || !(vatom_A3 > 0)) return EHC_E_INVAL;
  if (n > (int64_t)kNaMaxBlocks * kNaAtomsPerBlock) return EHC_E_INVAL;   // beyond the fixed scratch
  double *part = nullptr;
  int r = scratch_ptr(&part);
  if (r != EHC_OK) return r;
  const double kB_J = 1.380649e-23, eV_J = 1.602176634e-19;
  const double cap = Ce_cap_kB > 0 ? Ce_cap_kB * kB_J / (vatom_A3 * 1e-30) : 0.0;
  const int nb = (int)((n + kNaAtomsPerBlock - 1) / kNaAtomsPerBlock);
  cudaStream_t st = (cudaStream_t)stream;
  // launched through cudaLaunchKernel so that each launch's own status is checked
  // (the thread's last-error slot may hold an unrelated earlier failure)
  if (nb > 0) {
    const double *T = Te_dev;
    double g = gamma_Ce, cp = cap;
    void *args[] = {&n, (void *)&T, &g, &cp, &part};
    if (cudaLaunchKernel((const void *)na_partial, dim3(nb), dim3(kNaThreads), args, 0, st) != cudaSuccess)
      return EHC_E_CUDA;
  }
  int nbi = nb;
  double esc = vatom_A3 * 1e-30 / eV_J;
  void *fargs[] = {&nbi, &part, &esc, &out_dev};
  if (cudaLaunchKernel((const void *)na_final, dim3(1), dim3(kNaThreads), fargs, 0, st) != cudaSuccess)
    return EHC_E_CUDA;
  return EHC_OK;
}
