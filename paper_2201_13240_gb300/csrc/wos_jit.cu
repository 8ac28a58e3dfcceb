// wos_jit.cu -- problem-specialised walk kernels, compiled at run time with NVRTC.
//
// Every step of the walk of Supplemental Algorithm 1 evaluates alpha, Phi, sigma,
// the source and (at the end) g, with the value, gradient and Laplacian that the
// transformation of Sec. 4.1 and App. A needs (sigma' = sigma/alpha + Lap gamma +
// |grad gamma|^2, f' = e^gamma f / alpha).  The generic kernel reads these fields
// from the problem's descriptors: a loop over separable terms with a warp-uniform
// branch per atom.  Here the fields of ONE problem are written out as C++ with its
// constants as literals, placed after the walk kernel's own headers and compiled
// for sm_103a, so that the compiler folds constants, drops the derivatives a call
// site does not use and shares sub-expressions between fields.  The domain, grid
// fields, the Green's-function step and the accumulation are the same source as
// the generic kernel (the headers are embedded in this library at build time).
//
// libnvrtc is opened with dlopen: a library without it still loads, and
// specialisation then fails with WOS_EUNSUPPORTED and a message.
#include <dlfcn.h>
#include <nvrtc.h>  // types and status codes only

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "wos.h"
#include "wos_internal.h"
#include "wos_jit.h"
#include "wos_problem.cuh"

// kJitHeaderNames / kJitHeaderTexts / kJitHeaderCount: the walk kernel's headers
#include "wos_jit_sources.inc"

namespace wos {
namespace {

// ---------------------------------------------------------------------------
// generated fields
// ---------------------------------------------------------------------------
std::string lit(double v) {
  char b[64];
  std::snprintf(b, sizeof b, "R(%a)", v);
  return b;
}

struct AtomCode {
  std::string h, d, e;  // value, first and second derivative (expressions)
  bool e_zero = false;
};

// one atom h(k x + phi) of term n on axis i: declarations into `out`, names into `a`
void gen_atom(std::string& out, int n, int i, int type, double k, double ph, AtomCode* a) {
  const std::string sfx = std::to_string(n) + "_" + std::to_string(i);
  const std::string x = "x" + std::to_string(i);
  const std::string t = "t" + sfx;
  if (k == 1.0 && ph == 0.0) out += "    const R " + t + " = " + x + ";\n";
  else out += "    const R " + t + " = " + lit(k) + " * " + x + " + " + lit(ph) + ";\n";
  const std::string h = "h" + sfx, d = "d" + sfx, e = "e" + sfx;
  switch (type) {
    case A_SIN:
    case A_COS: {
      out += "    R s" + sfx + ", c" + sfx + ";\n    w_sincos(" + t + ", &s" + sfx + ", &c" + sfx + ");\n";
      const std::string s = "s" + sfx, c = "c" + sfx;
      if (type == A_SIN) {
        a->h = s;
        a->d = "(" + lit(k) + " * " + c + ")";
        a->e = "(" + lit(-k * k) + " * " + s + ")";
      } else {
        a->h = c;
        a->d = "(" + lit(-k) + " * " + s + ")";
        a->e = "(" + lit(-k * k) + " * " + c + ")";
      }
      return;
    }
    case A_EXP:
      out += "    const R " + h + " = w_exp(" + t + ");\n";
      a->h = h;
      a->d = "(" + lit(k) + " * " + h + ")";
      a->e = "(" + lit(k * k) + " * " + h + ")";
      return;
    case A_SINH:
    case A_COSH: {
      out += "    const R x" + sfx + " = w_exp(" + t + "), y" + sfx + " = w_div(R(1), x" + sfx + ");\n";
      out += "    const R sh" + sfx + " = R(0.5) * (x" + sfx + " - y" + sfx + "), ch" + sfx + " = R(0.5) * (x" + sfx +
             " + y" + sfx + ");\n";
      const std::string sh = "sh" + sfx, ch = "ch" + sfx;
      const std::string& v = (type == A_SINH) ? sh : ch;
      const std::string& w = (type == A_SINH) ? ch : sh;
      a->h = v;
      a->d = "(" + lit(k) + " * " + w + ")";
      a->e = "(" + lit(k * k) + " * " + v + ")";
      return;
    }
    case A_LIN:
      a->h = t;
      a->d = lit(k);
      a->e = "R(0)";
      a->e_zero = true;
      return;
    case A_QUAD:
      a->h = "(" + t + " * " + t + ")";
      a->d = "(" + lit(2.0 * k) + " * " + t + ")";
      a->e = lit(2.0 * k * k);
      return;
    default:
      a->h = "R(1)";
      a->d = "R(0)";
      a->e = "R(0)";
      a->e_zero = true;
      return;
  }
}

// c prod_i h_i(k_i x_i + phi_i), summed over the field's terms (the generic sst_eval)
void gen_sst(std::string& out, const DevProblem<double>& P, const DevField<double>& F, int dim) {
  for (int n = 0; n < F.nterms; ++n) {
    const DevTerm<double>& T = P.terms[F.first + n];
    out += "    // term " + std::to_string(n) + "\n";
    std::vector<int> nc;
    AtomCode at[3];
    for (int i = 0; i < dim; ++i) {
      if (T.type[i] == A_ONE) continue;
      nc.push_back(i);
      gen_atom(out, n, i, T.type[i], T.k[i], T.phi[i], &at[i]);
    }
    const std::string c = lit(T.c);
    auto prod_except = [&](int skip) {
      std::string s;
      for (int i : nc) {
        if (i == skip) continue;
        s += " * " + at[i].h;
      }
      return s;
    };
    out += "    o.v += " + c + prod_except(-1) + ";\n";
    if (nc.empty()) continue;
    out += "    if (deriv) {\n";
    static const char* gname[3] = {"o.gx", "o.gy", "o.gz"};
    for (int j : nc) out += std::string("      ") + gname[j] + " += " + c + " * " + at[j].d + prod_except(j) + ";\n";
    for (int j : nc) {
      if (at[j].e_zero) continue;
      out += "      o.lap += " + c + " * " + at[j].e + prod_except(j) + ";\n";
    }
    out += "    }\n";
  }
}

void gen_field(std::string& out, const DevProblem<double>& P, const DevField<double>& F, const char* id,
               const char* member, int dim) {
  out += std::string("  case ") + id + ": {\n";
  switch (F.kind) {
    case F_CONST:
      out += "    o.v = " + lit(F.value) + ";\n";
      break;
    case F_SST:
      gen_sst(out, P, F, dim);
      break;
    case F_GRID_LINEAR:
      out += std::string("    const R x[3] = {x0, x1, x2};\n    o.v = grid_linear<DIM>(P.") + member + ", x);\n";
      break;
    case F_GRID_BSPLINE:
      out += "    const R x[3] = {x0, x1, x2};\n    R g[3] = {R(0), R(0), R(0)};\n";
      out += std::string("    grid_bspline<DIM>(P.") + member + ", x, &o.v, g, &o.lap, deriv);\n";
      out += "    o.gx = g[0];\n    o.gy = g[1];\n    o.gz = g[2];\n";
      break;
    default:  // ZERO; a MANUFACTURED source is never evaluated as a field
      break;
  }
  out += "    return o;\n  }\n";
}

// ---------------------------------------------------------------------------
// NVRTC, opened at run time
// ---------------------------------------------------------------------------
struct Nvrtc {
  bool ok = false;
  std::string why;
  const char* (*GetErrorString)(nvrtcResult);
  nvrtcResult (*CreateProgram)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*DestroyProgram)(nvrtcProgram*);
  nvrtcResult (*CompileProgram)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*GetProgramLogSize)(nvrtcProgram, size_t*);
  nvrtcResult (*GetProgramLog)(nvrtcProgram, char*);
  nvrtcResult (*GetCUBINSize)(nvrtcProgram, size_t*);
  nvrtcResult (*GetCUBIN)(nvrtcProgram, char*);
  nvrtcResult (*AddNameExpression)(nvrtcProgram, const char*);
  nvrtcResult (*GetLoweredName)(nvrtcProgram, const char*, const char**);
};

const Nvrtc& nvrtc() {
  static Nvrtc api;
  static std::once_flag once;
  std::call_once(once, [] {
    std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char* env : {"CUDA_HOME", "CUDA_PATH"}) {
      const char* h = std::getenv(env);
      if (h && *h) names.push_back(std::string(h) + "/lib64/libnvrtc.so.13");
    }
    names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    void* lib = nullptr;
    for (const std::string& n : names) {
      lib = dlopen(n.c_str(), RTLD_NOW | RTLD_LOCAL);
      if (lib) break;
    }
    if (!lib) {
      api.why = "libnvrtc.so.13 not found (needed to specialise a problem's walk kernel)";
      return;
    }
    bool all = true;
    auto sym = [&](const char* n) {
      void* p = dlsym(lib, n);
      if (!p) all = false;
      return p;
    };
    api.GetErrorString = reinterpret_cast<decltype(api.GetErrorString)>(sym("nvrtcGetErrorString"));
    api.CreateProgram = reinterpret_cast<decltype(api.CreateProgram)>(sym("nvrtcCreateProgram"));
    api.DestroyProgram = reinterpret_cast<decltype(api.DestroyProgram)>(sym("nvrtcDestroyProgram"));
    api.CompileProgram = reinterpret_cast<decltype(api.CompileProgram)>(sym("nvrtcCompileProgram"));
    api.GetProgramLogSize = reinterpret_cast<decltype(api.GetProgramLogSize)>(sym("nvrtcGetProgramLogSize"));
    api.GetProgramLog = reinterpret_cast<decltype(api.GetProgramLog)>(sym("nvrtcGetProgramLog"));
    api.GetCUBINSize = reinterpret_cast<decltype(api.GetCUBINSize)>(sym("nvrtcGetCUBINSize"));
    api.GetCUBIN = reinterpret_cast<decltype(api.GetCUBIN)>(sym("nvrtcGetCUBIN"));
    api.AddNameExpression = reinterpret_cast<decltype(api.AddNameExpression)>(sym("nvrtcAddNameExpression"));
    api.GetLoweredName = reinterpret_cast<decltype(api.GetLoweredName)>(sym("nvrtcGetLoweredName"));
    if (!all) {
      api.why = "libnvrtc lacks an expected symbol";
      return;
    }
    api.ok = true;
  });
  return api;
}

const char* kVariantName[kJitVariants] = {"plain", "weight window", "gradient"};

// the kernel of a variant: <DIM, R, MESH, BATCHED, WW, GRAD, DRIFT>
std::string kernel_expr(int dim, bool fp64, bool mesh, bool drift, int variant) {
  const bool ww = variant == kJitWindow, grad = variant == kJitGrad;
  return std::string("wos::wos_walk_spec_kernel<") + std::to_string(dim) + ", " + (fp64 ? "double" : "float") + ", " +
         (mesh ? "true" : "false") + ", false, " + (ww ? "true" : "false") + ", " + (grad ? "true" : "false") + ", " +
         (drift ? "true" : "false") + ">";
}

}  // namespace

std::string jit_source(const DevProblem<double>& P) {
  const int dim = P.dim;
  std::string s;
  s += "// walk kernel specialised to one problem (" + std::to_string(dim) + "D): generated field code\n";
  s += "#define WOS_JIT_FIELDS 1\n";
  s += "#define WOS_JIT_F_KIND " + std::to_string(P.f.kind) + "\n";
  // analytic domains: the kind and its parameters as constants (meshes and CSG lists keep
  // their descriptors)
  if (P.domain_kind == D_BOX || P.domain_kind == D_BALL || P.domain_kind == D_ANNULUS ||
      P.domain_kind == D_ROUNDED_BOX) {
    s += "#define WOS_JIT_DOMAIN_KIND " + std::to_string(P.domain_kind) + "\n";
    s += "#define WOS_JIT_DOMAIN_PARAMS {";
    for (int i = 0; i < 16; ++i) s += (i ? ", " : "") + lit(P.dom[i]);
    s += "}\n";
  }
  // resident blocks per SM: 3D 6 (80 registers; 7 blocks at 72 registers measured 0.6 %
  // slower, 8 at 64 registers 5 % slower), 2D 8 (64 registers), neither spills
  s += (dim == 3) ? "#define WOS_WALK_MIN_BLOCKS 6\n" : "#define WOS_WALK_MIN_BLOCKS 8\n";
  s += "#include \"wos_walk_impl.cuh\"\n#include \"wos_adjoint_impl.cuh\"\n\nnamespace wos {\n\n";
  s += "template <int DIM, typename R>\n";
  s += "__device__ __forceinline__ FieldVal<R> jit_field(const DevProblem<R>& P, int id, R x0, R x1, R x2, "
       "bool deriv) {\n";
  s += "  FieldVal<R> o = {R(0), R(0), R(0), R(0), R(0)};\n";
  s += "  switch (id) {\n";
  gen_field(s, P, P.alpha, "FLD_ALPHA", "alpha", dim);
  gen_field(s, P, P.phi, "FLD_PHI", "phi", dim);
  gen_field(s, P, P.sigma, "FLD_SIGMA", "sigma", dim);
  gen_field(s, P, P.f, "FLD_F", "f", dim);
  gen_field(s, P, P.g, "FLD_G", "g", dim);
  gen_field(s, P, P.um, "FLD_UM", "um", dim);
  static const char* om_id[3] = {"FLD_OMEGA0", "FLD_OMEGA0 + 1", "FLD_OMEGA0 + 2"};
  static const char* om_mem[3] = {"omega[0]", "omega[1]", "omega[2]"};
  for (int d = 0; d < dim; ++d) gen_field(s, P, P.omega[d], om_id[d], om_mem[d], dim);
  s += "  default:\n    return o;\n  }\n}\n\n}  // namespace wos\n";
  return s;
}

bool same_field(const DevProblem<double>& A, const DevField<double>& F, const DevProblem<double>& B,
                const DevField<double>& G) {
  if (F.kind != G.kind) return false;
  if (F.kind == F_CONST) return F.value == G.value;
  if (F.kind != F_SST) return true;  // ZERO; grids read the walk's own descriptor
  if (F.nterms != G.nterms) return false;
  for (int n = 0; n < F.nterms; ++n) {
    const DevTerm<double>& s = A.terms[F.first + n];
    const DevTerm<double>& t = B.terms[G.first + n];
    if (s.c != t.c) return false;
    for (int i = 0; i < 3; ++i)
      if (s.type[i] != t.type[i] || s.k[i] != t.k[i] || s.phi[i] != t.phi[i]) return false;
  }
  return true;
}

std::string jit_source_batch(const BatchJitInfo& info) {
  const DevProblem<double>& P = info.rep;
  const int dim = P.dim;
  std::string s;
  s += "// walk kernel specialised to a batch of problems (" + std::to_string(dim) +
       "D): fields shared by every problem are generated code, the others are interpreted\n";
  s += "#define WOS_JIT_FIELDS 1\n";
  s += "#define WOS_JIT_F_KIND " + std::to_string(P.f.kind) + "\n";
  s += (dim == 3) ? "#define WOS_WALK_MIN_BLOCKS 7\n" : "#define WOS_WALK_MIN_BLOCKS 8\n";
  s += "#include \"wos_walk_impl.cuh\"\n\nnamespace wos {\n\n";
  s += "template <int DIM, typename R>\n";
  s += "__device__ __forceinline__ FieldVal<R> jit_field(const DevProblem<R>& P, int id, R x0, R x1, R x2, "
       "bool deriv) {\n";
  s += "  FieldVal<R> o = {R(0), R(0), R(0), R(0), R(0)};\n";
  s += "  switch (id) {\n";
  const DevField<double>* fields[6] = {&P.alpha, &P.phi, &P.sigma, &P.f, &P.g, &P.um};
  static const char* ids[6] = {"FLD_ALPHA", "FLD_PHI", "FLD_SIGMA", "FLD_F", "FLD_G", "FLD_UM"};
  static const char* mem[6] = {"alpha", "phi", "sigma", "f", "g", "um"};
  for (int f = 0; f < 6; ++f) {
    if (info.uniform & (1u << f)) {
      gen_field(s, P, *fields[f], ids[f], mem[f], dim);
    } else {
      s += std::string("  case ") + ids[f] + ":\n    return field_eval<DIM>(P, P." + mem[f] +
           ", x0, x1, x2, deriv);\n";
    }
  }
  s += "  default:\n    return o;\n  }\n}\n\n}  // namespace wos\n";
  return s;
}

namespace {
std::string batch_kernel_expr(int dim, bool fp64, int minb) {
  return std::string("wos::wos_walk_spec_kernel<") + std::to_string(dim) + ", " + (fp64 ? "double" : "float") +
         ", false, true, false, false, false, " + std::to_string(minb) + ">";
}

// NVRTC compile of a source with the given kernel name expressions
int compile_exprs(const std::string& src, const std::vector<std::string>& exprs, std::vector<char>* cubin,
                  std::vector<std::string>* lowered, std::string* log) {
  const Nvrtc& api = nvrtc();
  if (!api.ok) {
    *log = api.why;
    return WOS_EUNSUPPORTED;
  }
  nvrtcProgram prog = nullptr;
  nvrtcResult r = api.CreateProgram(&prog, src.c_str(), "wos_walk_specialised.cu", kJitHeaderCount, kJitHeaderTexts,
                                    kJitHeaderNames);
  if (r != NVRTC_SUCCESS) {
    *log = std::string("nvrtcCreateProgram: ") + api.GetErrorString(r);
    return WOS_EUNSUPPORTED;
  }
  for (const std::string& e : exprs) {
    r = api.AddNameExpression(prog, e.c_str());
    if (r != NVRTC_SUCCESS) {
      *log = std::string("nvrtcAddNameExpression: ") + api.GetErrorString(r);
      api.DestroyProgram(&prog);
      return WOS_EUNSUPPORTED;
    }
  }
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo"};
  r = api.CompileProgram(prog, 3, opts);
  size_t ls = 0;
  api.GetProgramLogSize(prog, &ls);
  std::string plog(ls, '\0');
  if (ls > 0) api.GetProgramLog(prog, &plog[0]);
  while (!plog.empty() && plog.back() == '\0') plog.pop_back();
  if (r != NVRTC_SUCCESS) {
    *log = std::string("nvrtcCompileProgram: ") + api.GetErrorString(r) + "\n" + plog;
    api.DestroyProgram(&prog);
    return WOS_EUNSUPPORTED;
  }
  size_t n = 0;
  api.GetCUBINSize(prog, &n);
  cubin->assign(n, 0);
  api.GetCUBIN(prog, cubin->data());
  lowered->assign(exprs.size(), std::string());
  for (size_t v = 0; v < exprs.size(); ++v) {
    const char* ln = nullptr;
    if (api.GetLoweredName(prog, exprs[v].c_str(), &ln) == NVRTC_SUCCESS && ln) (*lowered)[v] = ln;
  }
  api.DestroyProgram(&prog);
  *log = plog;
  return WOS_OK;
}
}  // namespace

void batch_jit_info(const DevProblem<double>* probs, int n, BatchJitInfo* info) {
  info->rep = probs[0];
  info->uniform = 0x3fu;
  info->f_kind_uniform = true;
  const DevProblem<double>& A = probs[0];
  const DevField<double>* fa[6] = {&A.alpha, &A.phi, &A.sigma, &A.f, &A.g, &A.um};
  for (int i = 1; i < n; ++i) {
    const DevProblem<double>& B = probs[i];
    const DevField<double>* fb[6] = {&B.alpha, &B.phi, &B.sigma, &B.f, &B.g, &B.um};
    for (int f = 0; f < 6; ++f)
      if (!same_field(A, *fa[f], B, *fb[f])) info->uniform &= ~(1u << f);
    if ((A.f.kind == F_MANUFACTURED) != (B.f.kind == F_MANUFACTURED)) info->f_kind_uniform = false;
  }
}

int jit_compile_batch(const BatchJitInfo& info, bool fp64, std::vector<char>* cubin, std::vector<std::string>* lowered,
                      std::string* log) {
  if (!info.f_kind_uniform) {
    *log = "the problems of the batch differ in the kind of their source (manufactured or not)";
    return WOS_EUNSUPPORTED;
  }
  const std::vector<std::string> exprs = {batch_kernel_expr(info.rep.dim, fp64, 0),
                                          batch_kernel_expr(info.rep.dim, fp64, 8)};
  return compile_exprs(jit_source_batch(info), exprs, cubin, lowered, log);
}

int jit_specialise_batch(JitState* js, const BatchJitInfo& info, bool fp64, std::string* why) {
  const int p = fp64 ? 1 : 0;
  if (js->kernel[p][0] != nullptr && js->kernel[p][1] != nullptr) return WOS_OK;
  std::vector<char> cubin;
  std::vector<std::string> lowered;
  std::string log;
  int rc = jit_compile_batch(info, fp64, &cubin, &lowered, &log);
  if (rc != WOS_OK) {
    *why = log;
    return rc;
  }
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) {
    *why = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return WOS_ECUDA;
  }
  cudaKernel_t found[2] = {nullptr, nullptr};
  for (int v = 0; v < 2; ++v) {
    e = lowered[v].empty() ? cudaErrorSymbolNotFound : cudaLibraryGetKernel(&found[v], lib, lowered[v].c_str());
    if (e != cudaSuccess) {
      *why = std::string("cudaLibraryGetKernel(batch): ") + cudaGetErrorString(e);
      cudaGetLastError();
      cudaLibraryUnload(lib);
      return WOS_ECUDA;
    }
  }
  js->kernel[p][0] = found[0];
  js->kernel[p][1] = found[1];
  js->libs.push_back(lib);
  return WOS_OK;
}

int jit_compile(const DevProblem<double>& P, bool fp64, int variant_mask, std::vector<char>* cubin,
                std::vector<std::string>* lowered, std::string* log) {
  const Nvrtc& api = nvrtc();
  if (!api.ok) {
    *log = api.why;
    return WOS_EUNSUPPORTED;
  }
  const bool mesh = P.domain_kind == D_MESH, drift = P.has_drift != 0;
  const std::string src = jit_source(P);
  nvrtcProgram prog = nullptr;
  nvrtcResult r = api.CreateProgram(&prog, src.c_str(), "wos_walk_specialised.cu", kJitHeaderCount, kJitHeaderTexts,
                                    kJitHeaderNames);
  if (r != NVRTC_SUCCESS) {
    *log = std::string("nvrtcCreateProgram: ") + api.GetErrorString(r);
    return WOS_EUNSUPPORTED;
  }
  // walk variants at 0..kJitVariants-1, then the adjoint kernels (sigma pass 1, 2, alpha pass 1, 2)
  std::vector<std::string> exprs(kJitExprs);
  if (variant_mask & (1 << kJitAdjoint)) {
    const std::string t = std::to_string(P.dim) + ", " + (fp64 ? "double" : "float");
    for (int a = 0; a < 2; ++a)
      for (int pass = 1; pass <= 2; ++pass)
        exprs[kJitVariants + 2 * a + pass - 1] = "wos::wos_adjoint_spec_kernel<" + t + (a ? ", true, " : ", false, ") +
                                                 std::to_string(pass) + ">";
  }
  for (int v = 0; v < kJitExprs; ++v) {
    if (v < kJitVariants) {
      if (!(variant_mask & (1 << v))) continue;
      exprs[v] = kernel_expr(P.dim, fp64, mesh, drift, v);
    } else if (exprs[v].empty()) {
      continue;
    }
    r = api.AddNameExpression(prog, exprs[v].c_str());
    if (r != NVRTC_SUCCESS) {
      *log = std::string("nvrtcAddNameExpression: ") + api.GetErrorString(r);
      api.DestroyProgram(&prog);
      return WOS_EUNSUPPORTED;
    }
  }
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo"};
  r = api.CompileProgram(prog, 3, opts);
  size_t ls = 0;
  api.GetProgramLogSize(prog, &ls);
  std::string plog(ls, '\0');
  if (ls > 0) api.GetProgramLog(prog, &plog[0]);
  while (!plog.empty() && plog.back() == '\0') plog.pop_back();
  if (r != NVRTC_SUCCESS) {
    *log = std::string("nvrtcCompileProgram: ") + api.GetErrorString(r) + "\n" + plog;
    api.DestroyProgram(&prog);
    return WOS_EUNSUPPORTED;
  }
  size_t n = 0;
  api.GetCUBINSize(prog, &n);
  cubin->assign(n, 0);
  api.GetCUBIN(prog, cubin->data());
  lowered->assign(kJitExprs, std::string());
  for (int v = 0; v < kJitExprs; ++v) {
    if (exprs[v].empty()) continue;
    const char* ln = nullptr;
    if (api.GetLoweredName(prog, exprs[v].c_str(), &ln) == NVRTC_SUCCESS && ln) (*lowered)[v] = ln;
  }
  api.DestroyProgram(&prog);
  *log = plog;
  return WOS_OK;
}

int jit_specialise(JitState* js, const DevProblem<double>& P, bool fp64, int variant_mask, std::string* why) {
  // a drift problem walks with the plain variant only (no window, no gradient, no adjoint)
  if (P.has_drift && (variant_mask & ~(1 << kJitPlain))) {
    *why = "an extra drift (omega) works with the plain walk only";
    return WOS_EUNSUPPORTED;
  }
  if ((variant_mask & (1 << kJitAdjoint)) && P.domain_kind == D_MESH) {
    *why = "the adjoint kernels run on analytic domains";
    return WOS_EUNSUPPORTED;
  }
  const int p = fp64 ? 1 : 0;
  int need = 0;
  for (int v = 0; v < kJitVariants; ++v)
    if ((variant_mask & (1 << v)) && js->kernel[p][v] == nullptr) need |= 1 << v;
  if ((variant_mask & (1 << kJitAdjoint)) && js->adjoint[p][0][0] == nullptr) need |= 1 << kJitAdjoint;
  if (need == 0) return WOS_OK;
  std::vector<char> cubin;
  std::vector<std::string> lowered;
  std::string log;
  int rc = jit_compile(P, fp64, need, &cubin, &lowered, &log);
  if (rc != WOS_OK) {
    *why = log;
    return rc;
  }
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) {
    *why = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return WOS_ECUDA;
  }
  // every requested kernel is found before any is published: a failure leaves the state as it was
  cudaKernel_t found[kJitExprs] = {};
  for (int v = 0; v < kJitExprs; ++v) {
    if (!(need & (1 << (v < kJitVariants ? v : kJitAdjoint)))) continue;
    e = lowered[v].empty() ? cudaErrorSymbolNotFound : cudaLibraryGetKernel(&found[v], lib, lowered[v].c_str());
    if (e != cudaSuccess) {
      *why = std::string("cudaLibraryGetKernel(") + (v < kJitVariants ? kVariantName[v] : "adjoint") +
             "): " + cudaGetErrorString(e);
      cudaGetLastError();
      cudaLibraryUnload(lib);
      return WOS_ECUDA;
    }
  }
  for (int v = 0; v < kJitVariants; ++v)
    if (need & (1 << v)) js->kernel[p][v] = found[v];
  if (need & (1 << kJitAdjoint)) {
    for (int a = 0; a < 2; ++a)
      for (int q = 0; q < 2; ++q) js->adjoint[p][a][q] = found[kJitVariants + 2 * a + q];
  }
  js->libs.push_back(lib);
  return WOS_OK;
}

void jit_release(JitState* js) {
  for (cudaLibrary_t lib : js->libs) cudaLibraryUnload(lib);
  js->libs.clear();
  for (auto& row : js->kernel)
    for (auto& k : row) k = nullptr;
  for (auto& plane : js->adjoint)
    for (auto& row : plane)
      for (auto& k : row) k = nullptr;
}

}  // namespace wos
