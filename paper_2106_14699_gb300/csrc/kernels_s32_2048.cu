// two-term FP32 forward, column, pair-product and weighted-row kernels for transform size 2048.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<df32, 2048>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 2048>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 2048>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 2048>::tm_cols(int);
template cudaError_t Sized<df32, 2048>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 2048>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 2048>::rows_w_smem();
template cudaError_t Sized<df32, 2048>::rows_w_max_blocks(int*);
}
