// Run-time compilation of pointwise groups that contain user-defined stages.
//
// In the paper a skeleton's leaves are kernels the programmer writes (Section 2: the SCT leaves
// are user OpenCL kernels, compiled by the OpenCL runtime when the computation is built). The
// counterpart here: a user stage is CUDA C source of a per-pixel device function. The executor
// generates the source of one kernel that applies a whole group of pointwise stages (built-in and
// user) in registers, compiles it for the current GPU with NVRTC, loads it through the CUDA
// runtime's library API and keeps it for the life of the process, keyed by source text and device.
//
// NVRTC is opened with dlopen the first time a user stage is built, so the executor itself does not
// depend on it; nvrtc.h is included for the declarations only.
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "mrw_internal.h"

namespace mrw {
namespace {

struct Nvrtc {
  bool tried = false;
  void *lib = nullptr;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) error_string = nullptr;
};

std::mutex g_mu;  // guards g_nvrtc and g_cache
Nvrtc g_nvrtc;
std::map<std::pair<int, std::string>, cudaKernel_t> g_cache;

template <typename F>
bool sym(void *lib, const char *name, F *f) {
  *f = reinterpret_cast<F>(dlsym(lib, name));
  return *f != nullptr;
}

// Opens NVRTC (the CUDA toolkit's shared library) once; false if it is not installed.
bool open_nvrtc(std::string *err) {
  Nvrtc &n = g_nvrtc;
  if (n.tried) {
    if (!n.lib) *err = "NVRTC (libnvrtc.so) was not found: user-defined stages need the CUDA toolkit's NVRTC";
    return n.lib != nullptr;
  }
  n.tried = true;
  std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
  for (const char *env : {"CUDA_HOME", "CUDA_PATH"}) {
    const char *root = getenv(env);
    if (root && *root) names.push_back(std::string(root) + "/lib64/libnvrtc.so");
  }
  names.push_back("/usr/local/cuda/lib64/libnvrtc.so");
  for (const std::string &nm : names) {
    n.lib = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL);
    if (n.lib) break;
  }
  if (n.lib && sym(n.lib, "nvrtcCreateProgram", &n.create) && sym(n.lib, "nvrtcCompileProgram", &n.compile) &&
      sym(n.lib, "nvrtcGetProgramLogSize", &n.log_size) && sym(n.lib, "nvrtcGetProgramLog", &n.log) &&
      sym(n.lib, "nvrtcGetCUBINSize", &n.cubin_size) && sym(n.lib, "nvrtcGetCUBIN", &n.cubin) &&
      sym(n.lib, "nvrtcDestroyProgram", &n.destroy) && sym(n.lib, "nvrtcGetErrorString", &n.error_string))
    return true;
  if (n.lib) dlclose(n.lib);
  n.lib = nullptr;
  *err = "NVRTC (libnvrtc.so) was not found: user-defined stages need the CUDA toolkit's NVRTC";
  return false;
}

// Compiles `src` to a cubin for sm_<arch>a. On failure *err holds NVRTC's message and log.
bool compile(const std::string &src, int arch, std::vector<char> *cubin, std::string *err) {
  Nvrtc &n = g_nvrtc;
  nvrtcProgram prog = nullptr;
  nvrtcResult r = n.create(&prog, src.c_str(), "mrw_user_chain.cu", 0, nullptr, nullptr);
  if (r != NVRTC_SUCCESS) {
    *err = std::string("nvrtcCreateProgram: ") + n.error_string(r);
    return false;
  }
  const std::string arch_opt = "--gpu-architecture=sm_" + std::to_string(arch) + "a";
  const char *opts[] = {arch_opt.c_str(), "-std=c++17", "--device-as-default-execution-space"};
  r = n.compile(prog, 3, opts);
  size_t ls = 0;
  std::string log;
  if (n.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
    log.resize(ls);
    if (n.log(prog, &log[0]) != NVRTC_SUCCESS) log.clear();
    while (!log.empty() && (log.back() == '\0' || log.back() == '\n')) log.pop_back();
  }
  bool ok = r == NVRTC_SUCCESS;
  if (ok) {
    size_t cs = 0;
    ok = n.cubin_size(prog, &cs) == NVRTC_SUCCESS && cs > 0;
    if (ok) {
      cubin->resize(cs);
      ok = n.cubin(prog, cubin->data()) == NVRTC_SUCCESS;
    }
    if (!ok) *err = "NVRTC produced no cubin";
  } else {
    *err = std::string("the user stage source does not compile (") + n.error_string(r) + "): " + log;
  }
  n.destroy(&prog);
  return ok;
}

}  // namespace

bool jit_check(const std::string &src, int arch, std::string *err) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!open_nvrtc(err)) return false;
  std::vector<char> cubin;
  return compile(src, arch, &cubin, err);
}

bool jit_kernel(const std::string &src, const char *entry, int device, int arch, cudaKernel_t *kernel,
                std::string *err) {
  std::lock_guard<std::mutex> lk(g_mu);
  const auto key = std::make_pair(device, src);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *kernel = it->second;
    return true;
  }
  if (!open_nvrtc(err)) return false;
  std::vector<char> cubin;
  if (!compile(src, arch, &cubin, err)) return false;
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e == cudaSuccess) e = cudaLibraryGetKernel(kernel, lib, entry);
  if (e != cudaSuccess) {
    *err = std::string("loading the compiled user-stage kernel: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return false;
  }
  g_cache.emplace(key, *kernel);  // the library stays loaded for the life of the process
  return true;
}

}  // namespace mrw
