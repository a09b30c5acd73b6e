// Host side of the TMA path: tensor-map encoding through the driver entry
// point (resolved once), and a cache of the maps of the ghosted node and
// element arrays keyed by base address and shape.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "modal.cuh"
#include "modal2.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace topo {

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// base, kind, pitch, ny, nz, box width, box rows, designs, design stride
using Key = std::tuple<const void*, int, int, int, int, int, int, int, long long>;
std::mutex g_mu;
std::map<Key, CUtensorMap> g_cache;

// kind 0: node vector (x, y, z, component, design); kind 1: element array
// (x, y, z, design).  The design dimension has all bt.designs() entries of
// the batch, bt.S bytes apart (a launch over a subset of the designs reads
// them by design index; one design: the dimension has one entry).
bool cached_map(const void* base, int kind, const Dims& d, int box_x, int box_y, const Bat& bt,
                CUtensorMap* out) {
  // one design: the natural size of the array (the dimension has one entry)
  const int nd = bt.designs();
  const long long natural = kind ? d.ecount * 4 : 3 * d.comp * 4;
  const long long dstride = (nd > 1) ? bt.S : natural;
  if (nd > 1 && (bt.S < natural || bt.S % 16 != 0)) return false;
  const Key key{base, kind, kind ? d.ex : d.px, d.ny, d.nz, box_x, box_y, nd, dstride};
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *out = it->second;
    return true;
  }
  CUtensorMap m;
  bool ok;
  if (kind == 0) {  // node vector: (x, y, z, component, design)
    const uint64_t dims[5] = {(uint64_t)d.px, (uint64_t)(d.ny + 3), (uint64_t)(d.nz + 3), 3,
                              (uint64_t)nd};
    const uint64_t strides[4] = {(uint64_t)d.px * 4, (uint64_t)d.px * (d.ny + 3) * 4,
                                 (uint64_t)d.comp * 4, (uint64_t)dstride};
    const uint32_t box[5] = {(uint32_t)box_x, (uint32_t)box_y, 1, 3, 1};
    ok = encode_tiled_map(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base), dims,
                          strides, box);
  } else {  // element array: (x, y, z, design)
    const uint64_t dims[4] = {(uint64_t)d.ex, (uint64_t)(d.ny + 2), (uint64_t)(d.nz + 2),
                              (uint64_t)nd};
    const uint64_t strides[3] = {(uint64_t)d.ex * 4, (uint64_t)d.ex * (d.ny + 2) * 4,
                                 (uint64_t)dstride};
    const uint32_t box[4] = {(uint32_t)box_x, (uint32_t)box_y, 1, 1};
    ok = encode_tiled_map(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims,
                          strides, box);
  }
  if (!ok) return false;
  if (g_cache.size() > 4096) g_cache.clear();
  g_cache[key] = m;
  *out = m;
  return true;
}

}  // namespace

bool encode_tiled_map(CUtensorMap* map, CUtensorMapDataType dtype, int rank, void* base,
                      const uint64_t* dims, const uint64_t* strides_bytes, const uint32_t* box) {
  EncodeFn fn = encoder();
  if (!fn) return false;
  // the box must fit inside the tensor in every dimension for this library's use
  for (int r = 0; r < rank; ++r)
    if ((uint64_t)box[r] > dims[r]) return false;
  cuuint64_t gd[5];
  cuuint64_t gs[4];
  cuuint32_t bx[5], es[5];
  for (int r = 0; r < rank; ++r) {
    gd[r] = dims[r];
    bx[r] = box[r];
    es[r] = 1;
  }
  for (int r = 0; r < rank - 1; ++r) gs[r] = strides_bytes[r];
  const CUresult res =
      fn(map, dtype, (cuuint32_t)rank, base, gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return res == CUDA_SUCCESS;
}

bool stencil_maps(const float* x, const float* E, const Dims& d, CUtensorMap* xmap,
                  CUtensorMap* emap) {
  return cached_map(x, 0, d, kBoxX, kBoxYN, Bat{}, xmap) &&
         cached_map(E, 1, d, kBoxX, kBoxYE, Bat{}, emap);
}

bool modal_maps(const float* x, const float* E, const Dims& d, const Bat& bt, int ty,
                CUtensorMap* xmap, CUtensorMap* emap) {
  return cached_map(x, 0, d, kMBoxX, ty + 1, bt, xmap) && cached_map(E, 1, d, kMBoxX, ty, bt, emap);
}

bool pair_maps(const float* x, const float* E, const Dims& d, const Bat& bt, CUtensorMap* xmap,
               CUtensorMap* emap) {
  return cached_map(x, 0, d, kPBoxX, kPBoxNY, bt, xmap) &&
         cached_map(E, 1, d, kPBoxX, kPBoxEY, bt, emap);
}

bool modal_aux_map(const float* v, const Dims& d, const Bat& bt, int ty, CUtensorMap* map) {
  return v != nullptr && cached_map(v, 0, d, kMAuxX, ty - 1, bt, map);
}

bool pair_aux_map(const float* v, const Dims& d, const Bat& bt, CUtensorMap* map) {
  return v != nullptr && cached_map(v, 0, d, kPBoxX, kPAuxY, bt, map);
}

}  // namespace topo
