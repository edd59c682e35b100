// Tensor-map (TMA descriptor) encoding shared by the translation units that
// stage tiles with cp.async.bulk.tensor.  The maps are encoded through the
// runtime's driver entry point (the library links the CUDA runtime only).
#pragma once

#include <cuda.h>

#include <cstdint>

namespace qdpg {

// A 2-D tiled map over `base`: dim0 x dim1 elements of esize (4 or 8) bytes,
// dim0 contiguous, `row_bytes` between rows (a multiple of 16), box box0 x
// box1, out-of-bounds elements read as zero.  False if the driver entry
// point is unavailable or the encoding fails (base not 16-byte aligned,
// stride not a multiple of 16, box too large).
bool encode_map_2d(CUtensorMap* m, const void* base, int esize, uint64_t dim0, uint64_t dim1, uint64_t row_bytes,
                   uint32_t box0, uint32_t box1);

// A 3-D tiled map: dim0 x dim1 x dim2 elements, strides stride1 and stride2
// bytes (multiples of 16) for dims 1 and 2, box box0 x box1 x box2.
bool encode_map_3d(CUtensorMap* m, const void* base, int esize, uint64_t dim0, uint64_t dim1, uint64_t dim2,
                   uint64_t stride1, uint64_t stride2, uint32_t box0, uint32_t box1, uint32_t box2);

}  // namespace qdpg
