// cq_jit.cu -- row-mode kernels specialised to one query shape, compiled at
// run time with NVRTC.
//
// A query's shape is everything in its descriptor that the row kernel's
// control flow depends on: each referenced column's encoding, value width,
// bit width, bitmap slot and stage offset; each predicate's column, kind and
// evaluation width; each key's column and digit mapping; each aggregate's
// kind, column and accumulator layout; the tile and warp shape.  The shape
// is written out as a class of constexpr functions (JitShape) and compiled
// together with the library's own device headers into a kernel whose tile
// body is FastBody<JitShape> (cq_fast.cuh).  Literal values stay in the
// descriptor passed at launch, so one compiled kernel serves every query of
// the same shape.  Kernels are cached per process by their source text.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "cq_internal.h"

namespace cq {

// The device headers the kernel is compiled from (text of csrc/*.cuh, cq_desc.h
// and include/cq.h, embedded by the build), and stand-ins for the system
// headers they include, which NVRTC does not provide.
struct JitHeader {
  const char* name;
  const char* text;
};
#include "cq_jit_headers.inc"   // kJitHeaders[], kNumJitHeaders (generated by build.py)

static const char* const kStubStdint =
    "#pragma once\n"
    "typedef signed char int8_t; typedef unsigned char uint8_t;\n"
    "typedef short int16_t; typedef unsigned short uint16_t;\n"
    "typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t;\n"
    "typedef unsigned long long uintptr_t;\n";
static const char* const kStubClimits =
    "#pragma once\n"
    "#define INT_MAX 2147483647\n#define INT_MIN (-INT_MAX - 1)\n"
    "#define LLONG_MAX 9223372036854775807LL\n#define LLONG_MIN (-LLONG_MAX - 1LL)\n"
    "#define UINT_MAX 4294967295U\n";
static const char* const kStubTypeTraits =
    "#pragma once\n"
    "namespace std { template <class T, T v> struct integral_constant {\n"
    "  static constexpr T value = v; typedef T value_type;\n"
    "  __host__ __device__ constexpr operator value_type() const { return value; } }; }\n";
static const char* const kStubEmpty = "#pragma once\n";

bool jit_enabled() {
  const char* e = getenv("CQ_JIT");
  return !(e && e[0] == '0');
}

static void emit_fn(std::string& s, const char* name, const std::vector<long long>& v) {
  s += "  __host__ __device__ static constexpr int ";
  s += name;
  s += "(int i) { return ";
  char buf[64];
  for (size_t k = 0; k < v.size(); ++k) {
    snprintf(buf, sizeof(buf), "i == %zu ? %lld : ", k, v[k]);
    s += buf;
  }
  s += "0; }\n";
}

// Helper warps of the specialised kernel: one per bitmap column, at most two.
int jit_helpers(const QueryDesc& q) { return q.n_bitmaps >= 2 ? 2 : 1; }

// Source of the shape class and kernel for descriptor q run with ncw compute
// warps, gpw 32-row groups per warp and minb CTAs per SM.
static std::string shape_source(const QueryDesc& q, int ncw, int gpw, int minb) {
  std::string s;
  char buf[512];
  s += "#include \"cq_fast.cuh\"\nnamespace cq {\nstruct JitShape {\n";
  const int n = snprintf(buf, sizeof(buf),
           "  static constexpr int tile_rows = %u, n_preds = %u, n_pbm = %u, n_keys = %u, n_aggs = %u;\n"
           "  static constexpr int n_cols = %u, n_bitmaps = %u, n_row_cols = %u, stage_bytes = %u;\n"
           "  static constexpr bool one_group = %s, table_dense = %s, ghash = %s, line_mode = %s;\n",
           q.tile_rows, q.n_preds, q.n_pbm, q.n_keys, q.n_aggs, q.n_cols, q.n_bitmaps, q.n_row_cols, q.stage_bytes,
           (q.n_groups == 1 && !q.ghash) ? "true" : "false", q.table_dense ? "true" : "false",
           q.ghash ? "true" : "false", q.line_mode ? "true" : "false");
  if (n < 0 || n >= (int)sizeof(buf)) return std::string();   // (never: the text is bounded)
  s += buf;
  std::vector<long long> enc, v64, e64, bw, bslot, roff, soff, bcol(q.n_bitmaps, 0), rcol;
  for (int c = 0; c < q.n_cols; ++c) {
    const ColDesc& d = q.cols[c];
    enc.push_back(d.enc);
    v64.push_back(d.v64);
    e64.push_back(d.e64);
    bw.push_back(d.bw);
    bslot.push_back(d.bslot);
    roff.push_back(d.raw_is_offset);
    soff.push_back(d.stage_off);
    if (d.bslot != 0xFF && d.bslot < q.n_bitmaps) bcol[d.bslot] = c;
  }
  for (int i = 0; i < q.n_row_cols; ++i) rcol.push_back(q.row_cols[i]);
  emit_fn(s, "enc", enc);
  emit_fn(s, "v64", v64);
  emit_fn(s, "e64", e64);
  emit_fn(s, "bcol", bcol);
  emit_fn(s, "row_col", rcol);
  emit_fn(s, "bw", bw);
  emit_fn(s, "bslot", bslot);
  emit_fn(s, "raw_off", roff);
  emit_fn(s, "stage_off", soff);
  std::vector<long long> pcol, pkind, pn32, ppbm, pneg, pcl;
  for (int i = 0; i < q.n_preds; ++i) {
    pcol.push_back(q.preds[i].col);
    pkind.push_back(q.preds[i].kind);
    pn32.push_back(q.preds[i].n32);
    ppbm.push_back(q.preds[i].pbm);
    pneg.push_back(q.preds[i].neg);
    pcl.push_back(q.preds[i].clause);
  }
  emit_fn(s, "pcol", pcol);
  emit_fn(s, "pkind", pkind);
  emit_fn(s, "pn32", pn32);
  emit_fn(s, "ppbm", ppbm);
  emit_fn(s, "pneg", pneg);
  emit_fn(s, "pcl", pcl);
  std::vector<long long> kcol, kremap, kn32;
  for (int k = 0; k < q.n_keys; ++k) {
    kcol.push_back(q.keys[k].col);
    kremap.push_back(q.keys[k].remap);
    kn32.push_back(q.keys[k].n32);
  }
  emit_fn(s, "kcol", kcol);
  emit_fn(s, "kremap", kremap);
  emit_fn(s, "kn32", kn32);
  std::vector<long long> akind, acol, asw, awide, asw32, agw, ared32, aw32, an32, as32, asrc, aub;
  for (int i = 0; i < q.n_aggs; ++i) {
    const AggDesc& a = q.aggs[i];
    akind.push_back(a.kind);
    acol.push_back(a.col);
    asw.push_back(a.sw);
    awide.push_back(a.wide);
    asw32.push_back(a.sw32);
    agw.push_back(a.gw);
    ared32.push_back(a.red32);
    aub.push_back(a.ubits);
    aw32.push_back(a.w32);
    an32.push_back(a.n32);
    as32.push_back(a.s32);
    // the value read of an earlier aggregate on the same column is reused
    int src = i;
    auto plain = [](const AggDesc& x) {
      return x.kind == AK_SUM || x.kind == AK_MIN || x.kind == AK_MAX || x.kind == AK_SUM2;
    };
    const bool plain_kind = plain(a);
    for (int j = 0; j < i && plain_kind; ++j) {
      const AggDesc& b = q.aggs[j];
      if (plain(b) && b.col == a.col && b.n32 == a.n32) {
        src = j;
        break;
      }
    }
    asrc.push_back(src);
  }
  emit_fn(s, "akind", akind);
  emit_fn(s, "acol", acol);
  emit_fn(s, "asw", asw);
  emit_fn(s, "awide", awide);
  emit_fn(s, "asw32", asw32);
  emit_fn(s, "agw", agw);
  emit_fn(s, "ared32", ared32);
  emit_fn(s, "aw32", aw32);
  emit_fn(s, "an32", an32);
  emit_fn(s, "as32", as32);
  emit_fn(s, "asrc", asrc);
  emit_fn(s, "aub", aub);
  s += "};\n}  // namespace cq\n";
  const int nh = jit_helpers(q);
  snprintf(buf, sizeof(buf),
           "extern \"C\" __global__ void __launch_bounds__(%d, %d) cq_row_jit(const __grid_constant__ cq::QueryDesc q) {\n",
           (ncw + nh) * 32, minb);
  s += buf;
  s += "  const unsigned long long t_begin = q.tile0 + (unsigned long long)blockIdx.x * q.n_tiles / gridDim.x;\n"
       "  const unsigned long long t_end = q.tile0 + (unsigned long long)(blockIdx.x + 1) * q.n_tiles / gridDim.x;\n"
       "  if (t_begin >= t_end) return;\n";
  snprintf(buf, sizeof(buf),
           "  cq::row_range<%d, %d, cq::FastBody<cq::JitShape>, %d>(q, cq::carve(q), t_begin, t_end);\n}\n", ncw, gpw,
           nh);
  s += buf;
  return s;
}

struct JitKernel {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  uint64_t smem_set_mask = 0;   // devices on which the dynamic shared-memory limit was raised
  double compile_s = 0;
};

static std::mutex g_jit_mu;
static std::unordered_map<std::string, JitKernel*>* g_jit_cache = nullptr;
static double g_jit_total_s = 0;
static uint64_t g_jit_compiles = 0;

static int compile(const std::string& src, JitKernel* k, bool load = true) {
  if (src.empty()) return set_error(CQ_ERR_CUDA, "the specialised kernel's source could not be formed");
  std::vector<const char*> names, texts;
  for (int i = 0; i < kNumJitHeaders; ++i) {
    names.push_back(kJitHeaders[i].name);
    texts.push_back(kJitHeaders[i].text);
  }
  const char* stubs[][2] = {{"stdint.h", kStubStdint}, {"stddef.h", kStubEmpty},  {"cuda_runtime.h", kStubEmpty},
                            {"climits", kStubClimits}, {"type_traits", kStubTypeTraits}};
  for (auto& st : stubs) {
    names.push_back(st[0]);
    texts.push_back(st[1]);
  }
  nvrtcProgram prog;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "cq_row_jit.cu", (int)names.size(), texts.data(), names.data());
  if (r != NVRTC_SUCCESS) return set_error(CQ_ERR_CUDA, "nvrtcCreateProgram failed: %s", nvrtcGetErrorString(r));
  // CQ_JIT_LOG=1 prints the compiler's resource report (registers, spills)
  const char* log_env = getenv("CQ_JIT_LOG");
  const bool verbose = log_env && log_env[0] == '1';
  std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-default-device",
                                   "-DCQ_JIT=1"};
  if (verbose) opts.push_back("--ptxas-options=-v");
  const auto t0 = std::chrono::steady_clock::now();
  r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  k->compile_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    if (log.size() > 3000) log.resize(3000);
    return set_error(CQ_ERR_CUDA, "run-time compilation of the row kernel failed: %s\n%s", nvrtcGetErrorString(r),
                     log.c_str());
  }
  if (verbose) {
    size_t ln = 0;
    nvrtcGetProgramLogSize(prog, &ln);
    std::string log(ln, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    fprintf(stderr, "[cq jit] compiled in %.2f s\n%s\n", k->compile_s, log.c_str());
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  std::vector<char> cubin(n);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  if (!load) return CQ_OK;
  cudaError_t e = cudaLibraryLoadData(&k->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "loading the compiled row kernel failed: %s", cudaGetErrorString(e));
  e = cudaLibraryGetKernel(&k->kernel, k->lib, "cq_row_jit");
  if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "row kernel not found in the compiled module: %s", cudaGetErrorString(e));
  return CQ_OK;
}

// The specialised kernel for q's shape (compiled on first use), ready to
// launch on `device` with up to `smem_limit` bytes of dynamic shared memory.
int jit_row_kernel(const QueryDesc& q, int ncw, int gpw, int minb, int device, size_t smem_limit, const void** fn) {
  const std::string src = shape_source(q, ncw, gpw, minb);
  std::lock_guard<std::mutex> lk(g_jit_mu);
  if (!g_jit_cache) g_jit_cache = new std::unordered_map<std::string, JitKernel*>();
  JitKernel*& k = (*g_jit_cache)[src];
  if (!k) {
    JitKernel* nk = new JitKernel;
    const int rc = compile(src, nk);
    if (rc != CQ_OK) {
      delete nk;
      g_jit_cache->erase(src);
      return rc;
    }
    k = nk;
    g_jit_total_s += nk->compile_s;
    g_jit_compiles++;
    const char* log_env = getenv("CQ_JIT_LOG");
    if (log_env && log_env[0] == '1')
      fprintf(stderr, "[cq jit] shape: %d compute warps, %d groups per warp, %d CTAs per SM, %u-row tiles, %u B "
                      "shared, line mode %d\n", ncw, gpw, minb, q.tile_rows, q.smem_bytes, (int)q.line_mode);
  }
  if (device < 64 && !((k->smem_set_mask >> device) & 1ull)) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k->kernel),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit);
    if (e != cudaSuccess) return set_error(CQ_ERR_CUDA, "shared-memory limit of the row kernel: %s", cudaGetErrorString(e));
    k->smem_set_mask |= 1ull << device;
  }
  *fn = reinterpret_cast<const void*>(k->kernel);
  return CQ_OK;
}

cudaError_t launch_row_jit(const void* fn, const QueryDesc& q, unsigned grid, int ncw, cudaStream_t s) {
  void* args[] = {const_cast<QueryDesc*>(&q)};
  return cudaLaunchKernel(fn, dim3(grid), dim3((ncw + jit_helpers(q)) * 32), args, q.smem_bytes, s);
}

}  // namespace cq

namespace cq {
// Eight synthetic shapes that between them use every encoding, predicate
// kind, key mapping, aggregate layout and group domain (shared hash table,
// run lines, global hash table, single group, dense table) of the
// specialised body, with and without the warp pre-reduction and the serial
// walk of sorted keys; only compiled.
static void check_shape(uint32_t variant, QueryDesc* q) {
  // variants 6 and 7: sorted-data shapes taking the serial walk -- a filter
  // of pass bitmaps only, staged 32-bit keys and values, 32-bit reducible
  // aggregates; 6 with the run-line table and 8-row lanes, 7 with a dense
  // table and 16-row lanes (a 14-bit column)
  if (variant == 6 || variant == 7) {
    memset(q, 0, sizeof(*q));
    q->tile_rows = 8192;
    q->n_cols = 5; q->n_preds = 1; q->n_keys = 2; q->n_aggs = 5; q->n_bitmaps = 2; q->n_pbm = 1;
    q->n_row_cols = 3; q->row_cols[0] = 2; q->row_cols[1] = 3; q->row_cols[2] = 4;
    const uint8_t kbw = variant == 6 ? 4 : 14;
    q->stage_bytes = 8192u * (kbw + 8 + 12) / 8;
    auto col = [&](int i, uint8_t enc, uint8_t bw, uint8_t bslot, uint32_t soff) {
      ColDesc& c = q->cols[i];
      c.enc = enc; c.bw = bw; c.bslot = bslot; c.raw_is_offset = enc == ENC_RLE ? 0 : 1; c.stage_off = soff;
    };
    col(0, ENC_RLE, 0, 0, 0);
    col(1, ENC_RLE, 0, 1, 0);
    col(2, ENC_DICT, kbw, 0xFF, 0);
    col(3, ENC_PACKED, 8, 0xFF, 8192u * kbw / 8);
    col(4, ENC_PACKED, 12, 0xFF, 8192u * (kbw + 8) / 8);
    q->preds[0].col = 1; q->preds[0].kind = PK_RANGE; q->preds[0].n32 = 1; q->preds[0].pbm = 0;
    q->keys[0].col = variant == 6 ? 0 : 2; q->keys[0].n32 = 1;
    q->keys[1].col = variant == 6 ? 2 : 3; q->keys[1].n32 = 1;
    auto agg = [&](int i, uint8_t kind, uint8_t c, uint8_t sw32, uint8_t s32, uint8_t w32) {
      AggDesc& a = q->aggs[i];
      a.kind = kind; a.col = c; a.sw32 = sw32; a.s32 = s32; a.w32 = w32; a.red32 = kind == AK_SUM;
      a.n32 = kind != AK_COUNT; a.gw = (uint32_t)(1 + 3 * i);
    };
    agg(0, AK_SUM, 3, 1, 1, 0);
    agg(1, AK_SUM, 4, 2, 3, 0);
    agg(2, AK_MIN, 4, 4, 0, 1);
    agg(3, AK_MAX, 3, 5, 0, 1);
    agg(4, AK_COUNT, 0, 0, 0, 0);
    if (variant == 6) {
      q->n_groups = 160000; q->table_slots = 1024;
      q->line_mode = 1; q->line_log2 = 5; q->line_inner = 16; q->line_swz = 15;
    } else {
      q->n_groups = 1000; q->table_slots = 1024; q->table_dense = 1;
    }
    return;
  }
  // variants 4 and 5: variants 0 and 3 with the run-line table (key 0 on
  // the RLE column 0)
  if (variant == 4 || variant == 5) {
    check_shape(variant == 4 ? 0 : 3, q);
    q->line_mode = 1;
    q->line_log2 = 4;
    q->line_slot = 0;
    q->line_inner = 64;
    q->line_swz = 31;
    if (variant == 4) q->aggs[1].s32 = 3;   // split limb words
    return;
  }
  memset(q, 0, sizeof(*q));
  q->tile_rows = 8192;
  q->n_groups = 1000;
  q->table_slots = 1024;
  auto col = [&](int i, uint8_t enc, uint8_t v64, uint8_t bw, uint8_t bslot, uint8_t roff, uint32_t soff) {
    ColDesc& c = q->cols[i];
    c.enc = enc; c.v64 = v64; c.bw = bw; c.bslot = bslot; c.raw_is_offset = roff; c.stage_off = soff;
  };
  auto pred = [&](int i, uint8_t c, uint8_t kind, uint8_t n32, uint8_t pbm) {
    PredDesc& p = q->preds[i];
    p.col = c; p.kind = kind; p.n32 = n32; p.pbm = pbm;
  };
  auto key = [&](int i, uint8_t c, uint8_t remap, uint8_t n32) {
    KeyDesc& k = q->keys[i];
    k.col = c; k.remap = remap; k.n32 = n32;
  };
  auto agg = [&](int i, uint8_t kind, uint8_t c, uint8_t sw, uint8_t wide, uint8_t sw32, uint32_t gw, uint8_t red32,
                 uint8_t w32, uint8_t n32, uint8_t s32) {
    AggDesc& a = q->aggs[i];
    a.kind = kind; a.col = c; a.sw = sw; a.wide = wide; a.sw32 = sw32; a.gw = gw; a.red32 = red32; a.w32 = w32;
    a.n32 = n32; a.s32 = s32;
  };
  if (variant == 0 || variant == 3) {
    q->n_cols = 5; q->n_preds = 2; q->n_keys = 2; q->n_aggs = 5; q->n_bitmaps = 2;
    col(0, ENC_RLE, 0, 0, 0, 0, 0);
    col(1, ENC_DICT, 0, 14, 0xFF, 1, 0);
    col(2, ENC_INDEX, 1, 0, 1, 0, 0);
    col(3, ENC_PLAIN, 0, 0, 0xFF, 0, 14352);
    col(4, ENC_PACKED, 1, 20, 0xFF, 1, 47136);
    q->n_row_cols = 3; q->row_cols[0] = 1; q->row_cols[1] = 3; q->row_cols[2] = 4;
    q->stage_bytes = 47136 + 8192 * 20 / 8;
    pred(0, 1, PK_BITMAP, 1, 0xFF);
    pred(1, 3, PK_RANGE, 1, 0xFF);
    key(0, 0, 0, 1);
    key(1, 1, 1, 1);
    agg(0, AK_ISUM, 2, 0, 1, 0, 1, 0, 0, 0, 0);
    agg(1, AK_SUM, 4, 0, 0, 1, 4, 1, 0, 1, 1);
    agg(2, AK_MIN, 4, 2, 0, 2, 7, 0, 1, 1, 0);
    agg(3, AK_MAX, 4, 2, 0, 3, 8, 0, 1, 1, 0);
    agg(4, AK_COUNT, 0, 0, 0, 0, 0, 0, 0, 0, 0);
    if (variant == 3) {
      agg(0, AK_COUNT, 0, 0, 0, 0, 0, 0, 0, 0, 0);   // reducible across a warp
      q->aggs[1].ubits = 20;                         // packed prefix sums
    }
  } else {
    q->n_cols = 5; q->n_preds = 6; q->n_keys = 1; q->n_aggs = 7; q->n_bitmaps = 2; q->n_pbm = 1;
    if (variant == 1) {
      q->n_groups = 1u << 20; q->table_dense = 0; q->table_slots = 512; q->ghash = 1;
    } else {
      q->n_groups = 1; q->table_dense = 1; q->table_slots = 1;
    }
    col(0, ENC_RLE, 1, 0, 0, 0, 0);
    col(1, ENC_INDEX, 1, 0, 1, 0, 0);
    col(2, ENC_PLAIN, 1, 0, 0xFF, 0, 0);
    col(3, ENC_PACKED, 1, 64, 0xFF, 0, 65552);
    col(4, ENC_PACKED, 1, 40, 0xFF, 1, 131104);
    pred(0, 0, PK_RANGE, 0, 0);
    pred(1, 1, PK_LIST, 0, 0xFF);
    pred(2, 2, PK_NE, 0, 0xFF);
    pred(3, 3, PK_BITMAP, 0, 0xFF);
    pred(4, 4, PK_LIST, 0, 0xFF);
    pred(5, 0, PK_TRUE, 0, 0xFF);
    // OR clauses and complements: (NOT p1 OR p2) AND (p4 OR TRUE), p0 negated
    q->preds[0].neg = 1;
    q->preds[1].neg = 1;
    q->preds[1].clause = PC_MEMBER;
    q->preds[2].clause = PC_LAST;
    q->preds[4].clause = PC_MEMBER;
    q->preds[5].clause = PC_LAST;
    key(0, 3, 0, 0);
    agg(0, AK_SUM, 2, 0, 1, 0, 1, 0, 0, 0, 0);
    agg(1, AK_MIN, 3, 2, 0, 0, 4, 0, 0, 0, 0);
    agg(2, AK_MAX, 3, 3, 0, 0, 5, 0, 0, 0, 0);
    agg(3, AK_IMIN, 1, 4, 0, 1, 6, 0, 0, 0, 0);
    agg(4, AK_IMAX, 1, 5, 0, 2, 8, 0, 0, 0, 0);
    agg(5, AK_SUM, 0, 6, 0, 0, 10, 0, 0, 0, 0);
    agg(6, AK_SUM, 4, 7, 0, 0, 13, 1, 0, 0, 0);
    if (variant == 2) {   // sums of squares (VAR / STD) of a plain and of an index column
      q->aggs[5].kind = AK_SUM2;
      q->aggs[5].pair = 6;
      q->aggs[3].kind = AK_ISUM2;
      q->aggs[3].pair = 0;
    }
  }
}
}  // namespace cq

// Compile (without loading) one of the built-in check shapes: a test of the
// run-time compilation that needs no GPU.  *seconds receives the compile time.
extern "C" int cq_jit_check(uint32_t variant, double* seconds) {
  cq::clear_error();
  if (variant > 7) return cq::set_error(CQ_ERR_INVALID_ARG, "variant must be 0 .. 7");
  cq::QueryDesc q;
  cq::check_shape(variant, &q);
  cq::JitKernel k;
  // (28 compute warps for the heterogeneous-like shapes, 16 for the others;
  // variant 6 as the two-CTA shape, whose register budget is the tightest)
  const bool wide = variant == 0 || variant == 3 || variant == 4 || variant == 5 || variant == 7;
  const int rc = cq::compile(cq::shape_source(q, wide ? 28 : 16, wide ? 8 : 16, variant == 6 ? 2 : 1), &k, false);
  if (seconds) *seconds = k.compile_s;
  return rc;
}

// Number of specialised kernels compiled by this process and the seconds spent.
extern "C" int cq_jit_stats(uint64_t* compiles, double* seconds) {
  std::lock_guard<std::mutex> lk(cq::g_jit_mu);
  if (compiles) *compiles = cq::g_jit_compiles;
  if (seconds) *seconds = cq::g_jit_total_s;
  return CQ_OK;
}
