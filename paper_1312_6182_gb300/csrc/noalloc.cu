// gpspca_sweep_static: one fused single-unit sweep that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// sweep: code that must not call cudaMalloc while another framework's
// caching allocator has reserved the GPU's free memory, latency-bound loops
// where an allocation (which can synchronise the device) is not acceptable,
// and code running where allocation is forbidden (callbacks, destructors,
// tightly budgeted services).  This entry point keeps all of its scratch in
// statically sized device arrays that exist for as long as the library is
// loaded; the caller passes the matrix, the iterate and the output buffers.
//
// The work is the same fused sweep kernel the solver uses, followed by the
// deterministic partial-sum reduction and a one-block step that forms the
// objective and normalises y.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "aux.cuh"
#include "plan.h"

namespace gpspca {

// Largest p this entry point takes, and its scratch: per-cluster partials of
// y (up to 160 clusters x p floats), the iterate copy (p floats), objective
// and Gram partials fit in 6 MiB for p <= 8192.  Every GPU that loads the
// library holds the array until the process exits.
constexpr int kStaticMaxP = 8192;
constexpr size_t kStaticScratchBytes = size_t(6) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
static __device__ __align__(256) IO g_static_io_sweep;   // what the sweep reads/writes
static __device__ __align__(256) IO g_static_io_reduce;  // what the reduction reads/writes
static __device__ __align__(256) State g_static_state;

struct StaticPtrs {
  bool ready = false;
  unsigned char* scratch = nullptr;
  IO* io_sweep = nullptr;
  IO* io_reduce = nullptr;
  State* st = nullptr;
  int nsm = 0;
};

static std::mutex g_static_mu;
static StaticPtrs g_static_ptrs[64];

// Device addresses of the static arrays for the current device.  The names
// above are host-side stand-ins; only these addresses may be passed to a kernel.
static int static_setup(int dev, StaticPtrs** out) {
  if (dev < 0 || dev >= 64) return record_error(GPSPCA_EINVAL, "device ordinal out of range");
  StaticPtrs& s = g_static_ptrs[dev];
  if (!s.ready) {
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&s.scratch), g_static_scratch) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.io_sweep), g_static_io_sweep) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.io_reduce), g_static_io_reduce) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.st), g_static_state) != cudaSuccess) {
      cudaGetLastError();
      return record_error(GPSPCA_ECUDA, "cudaGetSymbolAddress failed for the static sweep scratch");
    }
    cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev);
    s.ready = true;
  }
  *out = &s;
  return GPSPCA_OK;
}

// Sets the non-finite bit when any entry of t is NaN or infinite: a NaN or
// infinity in A or x, or a product that overflowed, reaches t (a NaN entry
// would otherwise fail every threshold test and drop out of the objective).
__global__ void static_check_finite(const float* __restrict__ t, int64_t n, State* st) {
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    bad |= !isfinite(t[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->error, kErrNonFinite);
}

// Sum of the reduction blocks' partials (fixed order): objective f and ||y||^2, then
// x_next = y / ||y|| (all zero when y = 0).  One block.  A non-finite f or
// ||y||^2 sets the non-finite bit.
__global__ void static_sweep_finish(const dd* fpart, int nobj, const double* gpart, int nred, float* x_next, int p,
                                    double* objective, State* st) {
  __shared__ double s_g;
  if (threadIdx.x == 0) {
    dd f{0.0f, 0.0f};
    double g = 0.0;
    for (int b = 0; b < nobj; ++b) f = dd_add(f, fpart[2 * b]);
    for (int b = 0; b < nred; ++b) g += gpart[b];
    s_g = g;
    const double fv = dd_to_double(f);
    *objective = fv;
    if (!isfinite(fv) || !isfinite(g)) atomicOr(&st->error, kErrNonFinite);
  }
  __syncthreads();
  const float inv = (s_g > 0.0 && isfinite(s_g)) ? static_cast<float>(1.0 / sqrt(s_g)) : 0.0f;
  for (int r = threadIdx.x; r < p; r += blockDim.x) x_next[r] *= inv;
}

}  // namespace gpspca

using namespace gpspca;

extern "C" int gpspca_sweep_static(const gpspca_matrix* A, gpspca_form form, double gamma, const float* x,
                                   float* x_next, float* t, double* objective, void* cuda_stream) {
  if (!A || !x || !x_next || !t || !objective) return record_error(GPSPCA_EINVAL, "a pointer argument is NULL");
  if (form != GPSPCA_SL1 && form != GPSPCA_SL0)
    return record_error(GPSPCA_EINVAL, "gpspca_sweep_static takes the single-unit forms SL1 / SL0");
  if (A->dtype != GPSPCA_F32 || A->location != GPSPCA_DEVICE || !A->data)
    return record_error(GPSPCA_EINVAL, "gpspca_sweep_static takes a float32 matrix in device memory");
  if (A->p < 1 || A->n < 1 || A->ld < A->p || A->p > (1 << 30) || A->n > (1 << 30))
    return record_error(GPSPCA_EINVAL, "bad shape");
  if (!(gamma >= 0.0) || !std::isfinite(gamma)) return record_error(GPSPCA_EINVAL, "gamma must be finite and >= 0");
  if (A->p > kStaticMaxP) {
    char msg[160];
    snprintf(msg, sizeof(msg), "p = %lld exceeds the static sweep's maximum of %d rows (its fixed scratch)",
             static_cast<long long>(A->p), kStaticMaxP);
    return record_error(GPSPCA_EINVAL, msg);
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  std::lock_guard<std::mutex> lk(g_static_mu);  // one call at a time: every call shares the arrays
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return record_error(GPSPCA_ECUDA, "cudaGetDevice failed");
  StaticPtrs* sp = nullptr;
  int rc = static_setup(dev, &sp);
  if (rc != GPSPCA_OK) return rc;

  const bool fast = (reinterpret_cast<uintptr_t>(A->data) % 16 == 0) && ((A->ld * 4) % 16 == 0);
  Plan pl;
  if ((rc = make_plan(GPSPCA_F32, form, 1, A->p, A->n, A->ld, fast, sp->nsm, &pl))) return rc;
  const int p = pl.p, n = pl.n;
  // scratch layout: ypart [ncl][p] | xcopy [p] | fpart [nobj][2] | gpart [nred]
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t off_ypart = 0;
  const size_t off_x = up(off_ypart + sizeof(float) * static_cast<size_t>(pl.ncl) * p);
  const size_t off_f = up(off_x + sizeof(float) * static_cast<size_t>(p));
  const size_t off_g = up(off_f + sizeof(dd) * 2 * static_cast<size_t>(pl.nobj));
  const size_t need = up(off_g + sizeof(double) * static_cast<size_t>(pl.nred));
  if (need > kStaticScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "p = %d needs %zu bytes of static scratch (%d clusters x p floats); the maximum is %zu bytes", p, need,
             pl.ncl, kStaticScratchBytes);
    return record_error(GPSPCA_EINVAL, msg);
  }
  unsigned char* sc = sp->scratch;
  IO io = {};
  io.A = A->data;
  io.Y = const_cast<float*>(x);  // the sweep evaluates X = x * 1 (read only)
  io.X = sc + off_x;             // the sweep's copy of the iterate it evaluated
  io.T = t;
  io.ypart = sc + off_ypart;
  io.fpart = reinterpret_cast<dd*>(sc + off_f);
  io.gpart = reinterpret_cast<double*>(sc + off_g);
  io.mu[0] = 1.0;
  io.gamma_in[0] = gamma;
  IO io_r = io;
  io_r.Y = x_next;  // the reduction writes y here
  State st = {};
  st.k = 0;
  st.n_active = 1;
  st.active[0] = 1;
  st.gamma[0] = gamma;
  st.W[0] = 1.0;
  // everything the kernels read starts from these records; the partial
  // buffers are fully rewritten by every call
  if (cudaMemcpyAsync(sp->io_sweep, &io, sizeof(IO), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(sp->io_reduce, &io_r, sizeof(IO), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(sp->st, &st, sizeof(State), cudaMemcpyHostToDevice, stream) != cudaSuccess) {
    cudaGetLastError();
    return record_error(GPSPCA_ECUDA, "copying the sweep records failed");
  }
  const Pass& q = pl.passes[0];
  SweepArgs a{sp->io_sweep, sp->st, pl.ld, p, n, 1, form, 0, 1, pl.ps, q.W, q.S, pl.cols_per_cl, pl.fast, 0, q.ov};
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(pl.ncl * pl.C);
  cfg.blockDim = dim3(q.threads);
  cfg.dynamicSmemBytes = q.smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  if (cudaLaunchKernelExC(&cfg, q.k, args) != cudaSuccess) {
    cudaGetLastError();
    return record_error(GPSPCA_ECUDA, "sweep launch failed");
  }
  ReduceArgs ra{sp->io_reduce, sp->st, pl.ncl, 1, p, 0, 1, 0, 0, 1, n, form, pl.nred, pl.nobj};
  launch_reduce(4, ra, stream);
  static_check_finite<<<static_cast<int>(std::min<int64_t>((n + 255) / 256, 4 * static_cast<int64_t>(sp->nsm))),
                        256, 0, stream>>>(t, n, sp->st);
  static_sweep_finish<<<1, 256, 0, stream>>>(reinterpret_cast<const dd*>(sc + off_f), pl.nobj,
                                              reinterpret_cast<const double*>(sc + off_g), pl.nred, x_next, p,
                                              objective, sp->st);
  if (cudaGetLastError() != cudaSuccess) return record_error(GPSPCA_ECUDA, "reduction launch failed");
  int32_t err = 0;
  if (cudaMemcpyAsync(&err, &sp->st->error, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return record_error(GPSPCA_ECUDA, "sweep execution failed");
  }
  if (err & kErrNonFinite)
    return record_error(GPSPCA_ENONFINITE, "A or x has a non-finite entry (or t, the objective or ||A g|| overflowed)");
  if (err & kErrTimeout) return record_error(GPSPCA_ETIMEDOUT, "a device-side wait for a tile copy gave up");
  if (err & kErrLaunch) return record_error(GPSPCA_ECUDA, "internal: sweep launched with a tile wider than it reduces");
  return GPSPCA_OK;
}
