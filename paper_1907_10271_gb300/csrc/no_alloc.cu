// Allocation-free solve on caller-supplied fields.
//
// Some callers cannot call cudaMalloc: code that runs while another component owns
// all device memory (an inference or simulation server with its own pool), plugins
// whose host framework forbids raw device allocations, or latency-critical paths
// that must not pay for an allocation or the implicit synchronisation cudaFree
// brings. mlmc_solve_theta_static serves them: it needs no context and allocates
// nothing. Its workspace is one file-scope device array of kStaticScratchBytes
// that every GPU loading this library holds until the process exits; the caller
// passes the fields and the output buffers.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "context.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;                // guards g_static_addr
std::map<int, char*> g_static_addr;    // device ordinal -> device address of g_static_scratch
thread_local std::string g_static_error;   // last failure on the calling thread

bool device_accessible(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mlmc_status static_fail(mlmc_status s, const std::string& m) {
  g_static_error = m;
  return s;
}

}  // namespace

extern "C" {

// The message stays valid until the calling thread's next call of mlmc_solve_theta_static.
const char* mlmc_static_last_error(void) { return g_static_error.c_str(); }

mlmc_status mlmc_solve_theta_static(const mlmc_config* cfg, void* cuda_stream, int32_t mesh_level, int64_t n,
                                    const double* theta, double* q, int32_t* status) {
  if (!cfg) return static_fail(MLMC_ERR_INVALID_ARG, "null config");
  // the same checks mlmc_create applies to a configuration, except on the KL fields,
  // which this entry point does not read
  mlmc_config vc = *cfg;
  vc.kl_terms = 1;
  vc.kl_std = 0.0;
  vc.kl_corr = 1.0;
  const std::string why = mlmc::validate(vc);
  if (!why.empty()) return static_fail(MLMC_ERR_INVALID_ARG, why);
  bool ok = true;
  const mlmc::Invariants U = mlmc::invariants(*cfg, ok);
  if (!ok)
    return static_fail(MLMC_ERR_INVALID_ARG, "material constants do not give a positive definite plane-strain stiffness");
  if (mesh_level < 0 || mesh_level >= cfg->levels) return static_fail(MLMC_ERR_INVALID_ARG, "mesh level out of range");
  if (n < 0 || (n > 0 && (!theta || !q))) return static_fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  // device address of the scratch array, looked up once per device with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(MLMC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_static_mu);
    auto it = g_static_addr.find(dev);
    if (it == g_static_addr.end()) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        g_static_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return MLMC_ERR_CUDA;
      }
      it = g_static_addr.emplace(dev, static_cast<char*>(ptr)).first;
    }
    scratch = it->second;
  }
  // a context on the stack: no KL bases (the fields are given), workspace borrowed
  mlmc::Context c;
  c.cfg = *cfg;
  c.stream = static_cast<cudaStream_t>(cuda_stream);
  c.device = dev;
  c.U = U;
  // no CUDA graphs: capturing and instantiating one allocates, and a caller's stream
  // that is itself being captured cannot begin a second capture
  c.graphs = false;
  // front of the scratch: staged inputs and outputs; the rest: solver workspace
  const mlmc::LevelLayout m = c.mesh(mesh_level);
  const int64_t ne = n * m.n_el();
  mlmc::Arena front;
  front.base = scratch;
  front.cap = kStaticScratchBytes;
  front.borrowed = true;
  double* th64 = front.carve<double>(device_accessible(theta) ? 0 : ne);
  float* tr32 = front.carve<float>(c.mixed() ? 2 * ne : 0);
  double* tr64 = front.carve<double>(c.mixed() ? 0 : 2 * ne);
  double* qd = front.carve<double>(device_accessible(q) ? 0 : 2 * n);
  int* sd = front.carve<int>(status && !device_accessible(status) ? n : 0);
  const size_t front_bytes = (front.used + 255) & ~(size_t)255;
  if (front_bytes >= kStaticScratchBytes)
    return static_fail(MLMC_ERR_INVALID_ARG, "fields exceed the 32 MiB static scratch");
  c.solve_arena.base = scratch + front_bytes;
  c.solve_arena.cap = kStaticScratchBytes - front_bytes;
  c.solve_arena.borrowed = true;
  cudaStream_t st = c.stream;
  // after work is queued, a failing call waits for it, so that the next serialised
  // call cannot find kernels of this one still writing the scratch array
  auto fail_queued = [&](mlmc_status s, const std::string& m) {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return static_fail(s, m);
  };
  const double* th_dev = theta;
  if (!device_accessible(theta)) {
    if ((e = cudaMemcpyAsync(th64, theta, sizeof(double) * ne, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return fail_queued(MLMC_ERR_CUDA, std::string("copy in: ") + cudaGetErrorString(e));
    th_dev = th64;
  }
  double* q_dev = device_accessible(q) ? q : qd;
  int* s_dev = status ? (device_accessible(status) ? status : sd) : nullptr;
  mlmc_status s;
  if (c.mixed()) {
    if ((e = mlmc::launch_theta_to_trig2<float>(th_dev, ne, tr32, st)) != cudaSuccess)
      return fail_queued(MLMC_ERR_CUDA, cudaGetErrorString(e));
    std::vector<mlmc::SolveGroup<float>> g{{mesh_level, n, tr32, q_dev, s_dev, nullptr}};
    s = mlmc::solve_groups<float>(c, g);
  } else {
    if ((e = mlmc::launch_theta_to_trig2<double>(th_dev, ne, tr64, st)) != cudaSuccess)
      return fail_queued(MLMC_ERR_CUDA, cudaGetErrorString(e));
    std::vector<mlmc::SolveGroup<double>> g{{mesh_level, n, tr64, q_dev, s_dev, nullptr}};
    s = mlmc::solve_groups<double>(c, g);
  }
  if (s == MLMC_ERR_OOM)
    return fail_queued(MLMC_ERR_INVALID_ARG, "n = " + std::to_string(n) + " samples on a " + std::to_string(m.nx) +
                                                 " x " + std::to_string(m.ny) +
                                                 " mesh need more than the 32 MiB static scratch");
  if (s != MLMC_OK) return fail_queued(s, c.err);
  if (q_dev != q && (e = cudaMemcpyAsync(q, q_dev, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail_queued(MLMC_ERR_CUDA, std::string("copy out: ") + cudaGetErrorString(e));
  if (s_dev && s_dev != status &&
      (e = cudaMemcpyAsync(status, s_dev, sizeof(int) * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail_queued(MLMC_ERR_CUDA, std::string("copy out: ") + cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail_queued(MLMC_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  return MLMC_OK;
}

}  // extern "C"
