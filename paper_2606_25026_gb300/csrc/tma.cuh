// Tensor-memory-accelerator (TMA) tile copies for the strided passes.
//
// A strided pass works on tiles of T adjacent columns x N points of a field
// where point n of column c in batch b sits at data[b * bstride + c + n * S]
// (complex64 units).  Seen as FP32 values that is a 3D tensor
//   dim 0: 2 W floats (the live columns, contiguous),
//   dim 1: N points (stride 8 S bytes),
//   dim 2: the batches (stride 8 bstride bytes),
// and one box of (2 T floats, BR points, 1 batch) lands in shared memory as
// BR rows of T complex values: exactly the element-major tile the FFT stages
// use (tile[n * T + t]).  N > 256 takes N / BR boxes (a box spans at most 256
// points).  Columns at or past W read as zeros and are never written back, so
// a ragged last tile needs no special case.
//
// Completion of the loads arrives on an mbarrier (transaction bytes); the
// wait is bounded, and a timeout sets a status bit instead of hanging.  The
// stores are bulk groups issued by one thread after every thread's writes are
// fenced for the async proxy; that thread waits until the tile has been read
// before the CTA may exit.  The tensor map is encoded on the host per launch
// (a pure host call) and passed as a __grid_constant__ kernel parameter.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include "spe_internal.cuh"
#include "tc16.cuh"

namespace spe {

// points per box: N itself up to 256, else the largest divisor of N that fits
__host__ __device__ constexpr int tma_box_rows(int n)
{
    return n <= 256 ? n : (n % 256 == 0 ? 256 : (n % 192 == 0 ? 192 : 128));
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z,
                                            unsigned long long *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
        : "memory");
}

// one contiguous run of bytes (a multiple of 16, both addresses 16-byte aligned) into shared memory,
// completing on the mbarrier's transaction count
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((uint64_t)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tm, int x, int y, int z, const void *src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit_wait_read()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Host: the driver's tensor-map encoder, looked up once through the runtime (so that libspe does not
// link the driver library itself); null when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Host: the tensor map of a strided pass's tiles (T columns x N points), or false when the shape
// does not meet the TMA rules (16-byte aligned base and strides, at least one full tile of live
// columns) and the pass keeps its per-thread copies.
inline bool encode_spass_tmap(const SParams &p, int n, int tw, CUtensorMap *tm)
{
    if (!p.tma || p.W < tw || n < 8) return false;
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    if (((uintptr_t)p.data & 15) != 0 || ((p.S * 8) & 15) != 0 || ((p.bstride * 8) & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * p.W, (cuuint64_t)n, (cuuint64_t)p.batches};
    const cuuint64_t strides[2] = {(cuuint64_t)p.S * 8, (cuuint64_t)p.bstride * 8};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * tw), (cuuint32_t)tma_box_rows(n), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)p.data, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace spe
