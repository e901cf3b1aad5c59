// two-term FP32 forward, column, pair-product and weighted-row kernels for transform size 1024.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<df32, 1024>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 1024>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 1024>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 1024>::tm_cols(int);
template cudaError_t Sized<df32, 1024>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 1024>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 1024>::rows_w_smem();
template cudaError_t Sized<df32, 1024>::rows_w_max_blocks(int*);
}
