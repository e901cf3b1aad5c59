// two-term FP32 forward, column, pair-product and weighted-row kernels for transform sizes 16, 32, 64, 128, 256.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<df32, 16>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 16>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 16>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 16>::tm_cols(int);
template cudaError_t Sized<df32, 16>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 16>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 16>::rows_w_smem();
template cudaError_t Sized<df32, 16>::rows_w_max_blocks(int*);
template cudaError_t Sized<df32, 32>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 32>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 32>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 32>::tm_cols(int);
template cudaError_t Sized<df32, 32>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 32>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 32>::rows_w_smem();
template cudaError_t Sized<df32, 32>::rows_w_max_blocks(int*);
template cudaError_t Sized<df32, 64>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 64>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 64>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 64>::tm_cols(int);
template cudaError_t Sized<df32, 64>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 64>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 64>::rows_w_smem();
template cudaError_t Sized<df32, 64>::rows_w_max_blocks(int*);
template cudaError_t Sized<df32, 128>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 128>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 128>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 128>::tm_cols(int);
template cudaError_t Sized<df32, 128>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 128>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 128>::rows_w_smem();
template cudaError_t Sized<df32, 128>::rows_w_max_blocks(int*);
template cudaError_t Sized<df32, 256>::fwd_rows(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 256>::fwd_cols(const Geom&, const PipeArgs<df32>&, bool, cudaStream_t);
template cudaError_t Sized<df32, 256>::pair_cols(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template int Sized<df32, 256>::tm_cols(int);
template cudaError_t Sized<df32, 256>::tm_max_blocks(int*);
template cudaError_t Sized<df32, 256>::pair_rows_w(const Geom&, const PipeArgs<df32>&, cudaStream_t);
template size_t Sized<df32, 256>::rows_w_smem();
template cudaError_t Sized<df32, 256>::rows_w_max_blocks(int*);
}
