// Tensor maps (TMA descriptors) for the pipelined check kernel's row copies.
//
// A frame-interleaved buffer [rows][Fp] is described as a 2-D tensor of Fp
// columns (frames, the contiguous dimension) and `rows` rows; a box of
// {32 V frames, h rows} is one check's rows of one frame group (h = 1 for the
// posterior rows, gathered four at a time). Encoding runs on the host, writes
// a 128-byte descriptor and allocates nothing; descriptors are cached per
// thread, keyed by everything that defines them.
#include <cudaTypedefs.h>

#include <array>
#include <cstring>
#include <mutex>

#include "ldpc_pass.h"

namespace ldpc {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encoder() {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

struct MapKey {
    const void *base;
    int dtype;
    uint64_t cols, rows, row_bytes;
    uint32_t box_cols, box_rows;
    bool operator==(const MapKey &o) const {
        return base == o.base && dtype == o.dtype && cols == o.cols && rows == o.rows && row_bytes == o.row_bytes &&
               box_cols == o.box_cols && box_rows == o.box_rows;
    }
};

struct MapEntry {
    MapKey key{};
    CUtensorMap map{};
    uint64_t used = 0;
    bool valid = false;
};

}  // namespace

cudaError_t tensor_map_2d(CUtensorMap *out, int dtype, const void *base, uint64_t cols, uint64_t rows,
                          uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows) {
    thread_local std::array<MapEntry, 32> cache;
    thread_local uint64_t tick = 0;
    const MapKey key{base, dtype, cols, rows, row_bytes, box_cols, box_rows};
    MapEntry *slot = &cache[0];
    for (auto &e : cache) {
        if (e.valid && e.key == key) {
            e.used = ++tick;
            *out = e.map;
            return cudaSuccess;
        }
        if (!e.valid || e.used < slot->used) slot = &e;
    }
    std::call_once(g_encode_once, load_encoder);
    if (!g_encode) return cudaErrorNotSupported;
    // the copy engine's rules: 16-byte aligned base and row pitch, box rows
    // of a multiple of 16 bytes
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || rows == 0 || cols == 0)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    CUresult r = g_encode(&m, static_cast<CUtensorMapDataType>(dtype), 2, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    slot->key = key;
    slot->map = m;
    slot->used = ++tick;
    slot->valid = true;
    *out = m;
    return cudaSuccess;
}

}  // namespace ldpc
