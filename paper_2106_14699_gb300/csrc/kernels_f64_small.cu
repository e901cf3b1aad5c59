// FP64 forward, column, pair-product and weighted-row kernels for transform sizes 16, 32, 64, 128, 256.
#include "pipeline_impl.cuh"
namespace cmif {
template cudaError_t Sized<double, 16>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 16>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 16>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 16>::tm_cols(int);
template cudaError_t Sized<double, 16>::tm_max_blocks(int*);
template cudaError_t Sized<double, 16>::pair_rows_w(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 16>::rows_w_smem();
template cudaError_t Sized<double, 16>::rows_w_max_blocks(int*);
template cudaError_t Sized<double, 32>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 32>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 32>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 32>::tm_cols(int);
template cudaError_t Sized<double, 32>::tm_max_blocks(int*);
template cudaError_t Sized<double, 32>::pair_rows_w(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 32>::rows_w_smem();
template cudaError_t Sized<double, 32>::rows_w_max_blocks(int*);
template cudaError_t Sized<double, 64>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 64>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 64>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 64>::tm_cols(int);
template cudaError_t Sized<double, 64>::tm_max_blocks(int*);
template cudaError_t Sized<double, 64>::pair_rows_w(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 64>::rows_w_smem();
template cudaError_t Sized<double, 64>::rows_w_max_blocks(int*);
template cudaError_t Sized<double, 128>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 128>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 128>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 128>::tm_cols(int);
template cudaError_t Sized<double, 128>::tm_max_blocks(int*);
template cudaError_t Sized<double, 128>::pair_rows_w(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 128>::rows_w_smem();
template cudaError_t Sized<double, 128>::rows_w_max_blocks(int*);
template cudaError_t Sized<double, 256>::fwd_rows(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 256>::fwd_cols(const Geom&, const PipeArgs<double>&, bool, cudaStream_t);
template cudaError_t Sized<double, 256>::pair_cols(const Geom&, const PipeArgs<double>&, cudaStream_t);
template int Sized<double, 256>::tm_cols(int);
template cudaError_t Sized<double, 256>::tm_max_blocks(int*);
template cudaError_t Sized<double, 256>::pair_rows_w(const Geom&, const PipeArgs<double>&, cudaStream_t);
template size_t Sized<double, 256>::rows_w_smem();
template cudaError_t Sized<double, 256>::rows_w_max_blocks(int*);
}
