// zmc_user.cu — user-defined integrands (include/zmc_user.h): the registry,
// NVRTC compilation of the sampling kernel around the user's g, and the
// per-(N, M, precision, device) kernel cache.
//
// NVRTC is opened with dlopen on first use, so the library loads and runs the
// compiled-in registry on machines without it.  The kernel's headers are read
// from the csrc/ directory next to libzmc.so and handed to NVRTC as in-memory
// headers, with minimal <cstdint>/<stdint.h>/<stddef.h> stand-ins.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/zmc_user.h"
#include "zmc_internal.h"
#include "zmc_runtime.h"

namespace zmc {

// ------------------------------------------------------------------ NVRTC --
struct Nvrtc {
  void* h = nullptr;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

static std::mutex g_user_mu;
static Nvrtc g_nvrtc;
static bool g_nvrtc_tried = false;

static bool open_nvrtc(std::string* why) {
  if (g_nvrtc.h) return true;
  if (g_nvrtc_tried) {
    *why = "NVRTC could not be loaded";
    return false;
  }
  g_nvrtc_tried = true;
  const char* names[] = {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13",
                         "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"};
  for (const char* n : names) {
    g_nvrtc.h = dlopen(n, RTLD_NOW | RTLD_LOCAL);
    if (g_nvrtc.h) break;
  }
  if (!g_nvrtc.h) {
    *why = "NVRTC (libnvrtc.so.13) not found";
    return false;
  }
#define ZMC_SYM(field, sym)                                                   \
  g_nvrtc.field = reinterpret_cast<decltype(g_nvrtc.field)>(dlsym(g_nvrtc.h, #sym)); \
  if (!g_nvrtc.field) {                                                       \
    *why = "NVRTC lacks " #sym;                                               \
    dlclose(g_nvrtc.h);                                                       \
    g_nvrtc.h = nullptr;                                                      \
    return false;                                                             \
  }
  ZMC_SYM(create, nvrtcCreateProgram)
  ZMC_SYM(add_name, nvrtcAddNameExpression)
  ZMC_SYM(compile, nvrtcCompileProgram)
  ZMC_SYM(log_size, nvrtcGetProgramLogSize)
  ZMC_SYM(log, nvrtcGetProgramLog)
  ZMC_SYM(cubin_size, nvrtcGetCUBINSize)
  ZMC_SYM(cubin, nvrtcGetCUBIN)
  ZMC_SYM(lowered, nvrtcGetLoweredName)
  ZMC_SYM(destroy, nvrtcDestroyProgram)
#undef ZMC_SYM
  return true;
}

// The csrc/ directory next to this library.
static std::string csrc_dir() {
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&open_nvrtc), &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    const size_t slash = p.find_last_of('/');
    return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) + "/csrc/";
  }
  return "csrc/";
}

static bool read_file(const std::string& path, std::string* out) {
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  *out = ss.str();
  return true;
}

static const char* kStdStub =
    "#pragma once\n"
    "typedef signed char int8_t; typedef unsigned char uint8_t;\n"
    "typedef short int16_t; typedef unsigned short uint16_t;\n"
    "typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t;\n";  // size_t: NVRTC's own

struct UserIntegrand {
  std::string name, source;
  int n_min = 1, n_max = ZMC_MAX_N;
  bool has32 = false, has64 = false;
};

struct UserKernel {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
};

static std::vector<UserIntegrand> g_users;
static std::map<std::tuple<int, int, int, int, int>, UserKernel> g_kernels;

// Compile scan_kernel<N, UserF<N>, prec> for integrand u at (N, M).
static int compile_user(const UserIntegrand& u, int N, int M, int prec,
                        std::vector<char>* cubin, std::string* lowered, std::string* log) {
  std::string why;
  if (!open_nvrtc(&why)) return fail(ZMC_ENOTFOUND, "%s", why.c_str());
  const std::string dir = csrc_dir();
  const char* files[] = {"zmc_scan_kernel.cuh", "zmc_integrands.cuh", "zmc_philox.cuh",
                         "zmc_internal.h", "zmc_user_functor.cuh"};
  std::vector<std::string> hdr_src, hdr_name;
  for (const char* f : files) {
    std::string s;
    if (!read_file(dir + f, &s)) return fail(ZMC_ENOTFOUND, "kernel header %s%s missing",
                                             dir.c_str(), f);
    hdr_src.push_back(s);
    hdr_name.push_back(f);
  }
  std::string zh;
  if (!read_file(dir + "../../include/zmc.h", &zh) && !read_file(dir + "../include/zmc.h", &zh))
    return fail(ZMC_ENOTFOUND, "include/zmc.h not found next to the library");
  hdr_src.push_back(zh);
  hdr_name.push_back("../../include/zmc.h");
  for (const char* std_name : {"cstdint", "stdint.h", "stddef.h"}) {
    hdr_src.push_back(kStdStub);
    hdr_name.push_back(std_name);
  }
  std::ostringstream src;
  src << "#define ZMC_N " << N << "\n#define ZMC_M " << M << "\n"
      << "#include <cstdint>\n" << u.source << "\n"
      << "#include \"zmc_scan_kernel.cuh\"\n#include \"zmc_user_functor.cuh\"\n";
  const std::string text = src.str();
  std::vector<const char*> hs, hn;
  for (size_t i = 0; i < hdr_src.size(); ++i) {
    hs.push_back(hdr_src[i].c_str());
    hn.push_back(hdr_name[i].c_str());
  }
  nvrtcProgram prog;
  if (g_nvrtc.create(&prog, text.c_str(), "zmc_user.cu", static_cast<int>(hs.size()), hs.data(),
                     hn.data()) != NVRTC_SUCCESS)
    return fail(ZMC_EINVAL, "nvrtcCreateProgram failed");
  std::ostringstream expr;
  expr << "&zmc::scan_kernel<" << N << ", zmc::" << (prec == ZMC_FP64 ? "UserF64<" : "UserF32<")
       << N << ">, " << prec << ">";
  const std::string ex = expr.str();
  g_nvrtc.add_name(prog, ex.c_str());
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
  const nvrtcResult cr = g_nvrtc.compile(prog, 3, opts);
  size_t ls = 0;
  g_nvrtc.log_size(prog, &ls);
  log->assign(ls, '\0');
  if (ls) g_nvrtc.log(prog, &(*log)[0]);
  if (cr != NVRTC_SUCCESS) {
    g_nvrtc.destroy(&prog);
    return ZMC_EINVAL;
  }
  size_t cs = 0;
  g_nvrtc.cubin_size(prog, &cs);
  cubin->resize(cs);
  g_nvrtc.cubin(prog, cubin->data());
  const char* low = nullptr;
  g_nvrtc.lowered(prog, ex.c_str(), &low);
  *lowered = low ? low : "";
  g_nvrtc.destroy(&prog);
  return ZMC_OK;
}

bool is_user_integrand(int id) { return id >= ZMC_G_USER_BASE; }

int user_validate(const zmc_scan_desc* d) {
  std::lock_guard<std::mutex> lk(g_user_mu);
  const int k = d->integrand_id - ZMC_G_USER_BASE;
  if (k < 0 || k >= static_cast<int>(g_users.size()))
    return fail(ZMC_ENOTFOUND, "unknown integrand id %d", d->integrand_id);
  const UserIntegrand& u = g_users[k];
  if (d->N < u.n_min || d->N > u.n_max)
    return fail(ZMC_EINVAL, "user integrand %s takes N in [%d, %d]", u.name.c_str(), u.n_min,
                u.n_max);
  if (d->precision == ZMC_FP64 ? !u.has64 : !u.has32)
    return fail(ZMC_EINVAL, "user integrand %s defines no %s version", u.name.c_str(),
                d->precision == ZMC_FP64 ? "zmc_user_g64" : "zmc_user_g32");
  return ZMC_OK;
}

int user_info(int id, zmc_integrand_info* info) {
  std::lock_guard<std::mutex> lk(g_user_mu);
  const int k = id - ZMC_G_USER_BASE;
  if (k < 0 || k >= static_cast<int>(g_users.size()))
    return fail(ZMC_ENOTFOUND, "unknown integrand id %d", id);
  std::memset(info, 0, sizeof(*info));
  info->id = id;
  std::snprintf(info->name, sizeof(info->name), "%s", g_users[k].name.c_str());
  info->m_rule = 0;
  return ZMC_OK;
}

// Launch the user integrand's sampling kernel (compiling and loading it on
// first use for this (N, M, precision, device)).
int user_launch(const zmc_scan_desc* d, const ScanArgs& a, int block, int64_t grid,
                size_t smem, cudaStream_t stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int k = d->integrand_id - ZMC_G_USER_BASE;
  const auto key = std::make_tuple(k, d->N, d->M, d->precision, dev);
  UserKernel uk;
  {
    std::lock_guard<std::mutex> lk(g_user_mu);
    auto it = g_kernels.find(key);
    if (it != g_kernels.end()) {
      uk = it->second;
    } else {
      std::vector<char> cubin;
      std::string lowered, log;
      const int prec_t = d->precision == ZMC_FP64 ? ZMC_FP64 : d->precision;
      int rc = compile_user(g_users[k], d->N, d->M, prec_t, &cubin, &lowered, &log);
      if (rc != ZMC_OK)
        return rc == ZMC_EINVAL ? fail(rc, "user integrand compile failed:\n%.400s", log.c_str())
                                : rc;
      cudaError_t e = cudaLibraryLoadData(&uk.lib, cubin.data(), nullptr, nullptr, 0, nullptr,
                                          nullptr, 0);
      if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryLoadData(user integrand)");
      e = cudaLibraryGetKernel(&uk.kernel, uk.lib, lowered.c_str());
      if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryGetKernel(user integrand)");
      g_kernels[key] = uk;
    }
  }
  void* args[] = {const_cast<ScanArgs*>(&a)};
  cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(uk.kernel),
                                   dim3(static_cast<unsigned>(grid)), dim3(block), args, smem,
                                   stream);
  if (e != cudaSuccess) return cuda_fail(e, "user integrand launch");
  return ZMC_OK;
}

}  // namespace zmc

extern "C" int zmc_integrand_register(const char* name, const char* source, int n_min,
                                      int n_max, int* id) {
  using namespace zmc;
  clear_error();
  if (!name || !source || !id) return fail(ZMC_EINVAL, "NULL argument");
  if (n_min < 1 || n_max > ZMC_MAX_N || n_min > n_max)
    return fail(ZMC_EINVAL, "dimension range [%d, %d] outside [1, %d]", n_min, n_max, ZMC_MAX_N);
  UserIntegrand u;
  u.name = name;
  u.source = source;
  u.n_min = n_min;
  u.n_max = n_max;
  std::vector<char> cubin;
  std::string lowered, log32, log64;
  {
    std::lock_guard<std::mutex> lk(g_user_mu);
    if (g_users.size() >= ZMC_MAX_USER_INTEGRANDS)
      return fail(ZMC_ENOMEM, "at most %d user integrands", ZMC_MAX_USER_INTEGRANDS);
    int r32 = compile_user(u, n_min, 1, ZMC_FP32_KAHAN, &cubin, &lowered, &log32);
    if (r32 == ZMC_ENOTFOUND) return r32;
    int r64 = compile_user(u, n_min, 1, ZMC_FP64, &cubin, &lowered, &log64);
    u.has32 = r32 == ZMC_OK;
    u.has64 = r64 == ZMC_OK;
    if (!u.has32 && !u.has64)
      return fail(ZMC_EINVAL, "user integrand %s does not compile:\n%.1500s", name,
                  log32.c_str());
    g_users.push_back(u);
    *id = ZMC_G_USER_BASE + static_cast<int>(g_users.size()) - 1;
  }
  clear_error();
  return ZMC_OK;
}
