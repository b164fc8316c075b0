// dcm_distance_noalloc: the box-interface distance sweeps without any device
// allocation and without a dcm_ctx.
//
// Who needs it: code that must not call cudaMalloc at all, e.g. a host
// program whose device memory is owned by another allocator or framework
// (and that therefore cannot create a dcm_ctx, whose scratch is allocated by
// dcm_create), or code embedded in a plugin that is only handed device
// buffers.  Such a caller passes the inputs and the output and this call uses,
// as its only scratch, a fixed array compiled into the library.
//
// The scratch is one file-scope __device__ array of kNoAllocBytes bytes.
// Every GPU that loads this library holds it until the process exits.  It
// keeps the second Jacobi iterate (one real per density box) and the per-sweep
// change flags; calls that need more than kNoAllocBytes are rejected.
//
// Host code cannot use the array's name as a device address (in host code the
// name refers to a host-side shadow), so the device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made with that
// device current, and cached per device index.  The stream passed in must
// belong to the current device, and a cudaDeviceReset of a device invalidates
// the cached address (later calls on that device would write through a stale
// pointer), so a program that resets a device must not call this entry point
// on it again.  All calls share the one array and it keeps the contents of the
// last call: the flags are cleared at the start of every call, and two calls
// whose kernels overlap on the GPU (different streams, or different host
// threads) race on the array and give undefined results.  Like dcm_distance,
// the call waits on the stream between chunks of sweeps to test convergence.
#include <mutex>

#include "dcm_internal.cuh"

namespace {

constexpr int64_t kNoAllocBytes = (int64_t)8 << 20;  // 8 MiB: a 1M-box grid in FP64, 2M boxes in FP32
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once).
int noalloc_scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return DCM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DCM_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return DCM_OK;
}

template <typename R>
__device__ __forceinline__ R inf_of();
template <>
__device__ __forceinline__ float inf_of<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double inf_of<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

template <typename R>
__global__ void k_na_init(const uint8_t* __restrict__ s, const uint8_t* __restrict__ iface, int64_t nbox,
                          R* __restrict__ D0, R* __restrict__ D1) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  R v = (!s[b] || iface[b]) ? (R)0 : inf_of<R>();
  D0[b] = v;
  D1[b] = v;
}

// Jacobi sweep of the Godunov update (same update as dcm_distance).
template <typename R>
__global__ void k_na_sweep(const R* __restrict__ Din, R* __restrict__ Dout, int nx, int ny, int nz, R h, R r_grid,
                           int32_t* __restrict__ flags, int it) {
  if (it > 0 && flags[it - 1] == 0) return;
  int x = blockIdx.y * blockDim.x + threadIdx.x;
  int yz = blockIdx.x;
  if (x >= nx) return;
  int y = yz % ny, z = yz / ny;
  int64_t b = x + (int64_t)nx * yz;
  R cur = Din[b];
  if (cur == (R)0) return;
  int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
  R a0 = fmin(Din[row + xm], Din[row + xp]);
  R a1 = fmin(Din[x + nx * (ym + (int64_t)ny * z)], Din[x + nx * (yp + (int64_t)ny * z)]);
  R a2 = fmin(Din[x + nx * (y + (int64_t)ny * zm)], Din[x + nx * (y + (int64_t)ny * zp)]);
  R t;
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  R d = a0 + h;
  if (d > a1) {
    R df = a0 - a1;
    d = (R)0.5 * (a0 + a1 + sqrt((R)2 * h * h - df * df));
    if (d > a2) {
      R sa = a0 + a1 + a2;
      R sq = a0 * a0 + a1 * a1 + a2 * a2;
      R disc = sa * sa - (R)3 * (sq - h * h);
      d = (sa + sqrt(disc > (R)0 ? disc : (R)0)) / (R)3;
    }
  }
  R out = cur;
  if (d < cur && d <= r_grid) {
    out = d;
    flags[it] = 1;
  }
  Dout[b] = out;
}

__global__ void k_na_finish(const int32_t* flags, int sweeps, int32_t* iters) {
  int first = -1;
  for (int k = 0; k < sweeps; ++k)
    if (flags[k] == 0) {
      first = k;
      break;
    }
  if (iters) *iters = first >= 0 ? first + 1 : -1;
}

template <typename R>
int na_distance(const dcm_params& p, const int64_t* nh, const uint8_t* s, const uint8_t* iface, R* D, int32_t* iters,
                cudaStream_t st, unsigned char* scratch) {
  int nx = (int)nh[0], ny = (int)nh[1], nz = (int)nh[2];
  int64_t nbox = nh[0] * nh[1] * nh[2];
  R* D1 = (R*)scratch;
  int64_t off = ((int64_t)sizeof(R) * nbox + 255) / 256 * 256;
  int32_t* flags = (int32_t*)(scratch + off);
  int iter_max = p.iter_max;
  double ramp = p.ramp > 0.0 ? p.ramp : p.rc_max - p.rc_min;
  R h = (R)p.h, rg = (R)(p.r_grid > 0.0 ? p.r_grid : ramp + 2.0 * p.h);
  if (cudaMemsetAsync(flags, 0, sizeof(int32_t) * (size_t)(iter_max + 2), st) != cudaSuccess) return DCM_ERR_CUDA;
  R* buf[2] = {D, D1};
  k_na_init<R><<<(unsigned)((nbox + 255) / 256), 256, 0, st>>>(s, iface, nbox, buf[0], buf[1]);
  dim3 grid((unsigned)(ny * nz), (unsigned)((nx + 127) / 128));
  int done = 0;
  bool converged = false;
  while (done < iter_max && !converged) {
    int m = iter_max - done < 8 ? iter_max - done : 8;
    for (int k = 0; k < m; ++k, ++done)
      k_na_sweep<R><<<grid, 128, 0, st>>>(buf[done & 1], buf[(done + 1) & 1], nx, ny, nz, h, rg, flags, done);
    int32_t last = 1;  // pageable host copy: no pinned allocation
    if (cudaMemcpyAsync(&last, flags + done - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return DCM_ERR_CUDA;
    converged = last == 0;
  }
  k_na_finish<<<1, 1, 0, st>>>(flags, done, iters);
  if (!converged && (done & 1))
    if (cudaMemcpyAsync(D, buf[1], sizeof(R) * nbox, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return DCM_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return DCM_ERR_CUDA;
  return converged ? DCM_OK : DCM_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" int dcm_distance_noalloc(const dcm_params* p, const uint8_t* s, const uint8_t* iface, void* D,
                                    int32_t* iters, dcm_stream_t stream) {
  if (!p || !s || !iface || !D) return DCM_ERR_INVALID_ARG;
  int r = dcm_validate_params(p, nullptr, 0);
  if (r) return r;
  int64_t nh[3];
  if (dcm_grid_dims(p, nullptr, nh) != DCM_OK) return DCM_ERR_BOX;
  int64_t nbox = nh[0] * nh[1] * nh[2];
  int64_t rsize = p->precision == DCM_PREC_FP64 ? 8 : 4;
  int64_t need = (rsize * nbox + 255) / 256 * 256 + 4 * ((int64_t)p->iter_max + 2);
  if (need > kNoAllocBytes) return DCM_ERR_CAPACITY;  // grid or iter_max too large for the fixed scratch
  void* scratch = nullptr;
  if ((r = noalloc_scratch_address(&scratch))) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->precision == DCM_PREC_FP64)
    return na_distance<double>(*p, nh, s, iface, (double*)D, iters, st, (unsigned char*)scratch);
  return na_distance<float>(*p, nh, s, iface, (float*)D, iters, st, (unsigned char*)scratch);
}
