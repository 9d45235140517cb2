// Tensor-core (tcgen05) GEMM of the mixed build: operand planes and launcher.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Three fp16 fixed-point slices of one GEMM operand, each a TMA tensor map
// over [batch][rows][ld] (32-element K boxes, 128 rows, 64B swizzle); an
// operand converted inside the GEMM uses map[0] only (an FP32 map).
struct TcOperand {
  alignas(64) unsigned char map[3][128];
};

// Encode the map of one fp16 plane: `rows` x `cols` valid elements per batch,
// leading dimension `ld` elements (ld * 2 bytes must be a multiple of 16).
cudaError_t make_plane_map(void* map_out, const void* base, int batch, int rows, int cols, int ld);

// out[b][m][n] (n < Nr real columns, interleaved complex) = A'[b] B'[b]^T for
// sliced operands: A' has M rows with exponents eA[b * seA + m], B' has Nr rows
// whose pair (2j, 2j + 1) shares the exponent eB[b * seB + j]; Kr real K.
// FP32 output, or FP64 output when out_f64.  K is taken in the chunks
// tc_chunk_blocks gives; with more than one chunk ps0 / pbc (tc_partial_elems
// elements each) hold the exact chunk sums until they are combined.  `err`
// receives a nonzero code if a device wait gave up.  gemm_done (may be null)
// is recorded on `s` right after the GEMM kernel, before any combine kernel,
// so that the GEMM alone can be timed.  products: 6 or 8 slice products per
// real product (about 2^-27 or 2^-30 of the row scales dropped).  a_conv: 0 =
// A is three planes; 1 = A.map[0] is an FP32 map (make_f32_map) of the
// interleaved complex A [rows][K], cut into its slices inside the kernel with
// the row exponents eA; 2 = A.map[0] is an FP32 map (make_f32_map_t) of the
// stored transpose [K][rows] of A; 3 = as 1, and A.map[1] an fp16 plane map
// (make_plane_map) of A's remainders below its FP32 values, each an fp16
// multiple q of its value's unit in the last place (q 2^(e - 24) for a value
// m 2^e, 1/2 <= m < 1), sliced with them.  herm (1 or 2): the product is Hermitian
// (B built from conj(A), Nr = 2 M, one K chunk, FP32 output): only the tiles
// that reach the diagonal are computed, and each writes its values on or
// above the diagonal, and with herm = 1 also their conjugates at the mirrored
// positions (herm = 2 leaves the part below the diagonal unwritten).
// dot_with (optional): when the product is split along K and its FP32 result
// is contiguous ([batch][M][Nr], ldo = Nr), the combine kernel also writes
// block partial sums of sum conj(w) out for w = dot_with of the same layout
// (2 doubles per block, at most dot_max blocks, into dot_partial) and sets
// *dot_blocks to their count; otherwise *dot_blocks = 0 and nothing is summed.
// b0: the product is entries b0 .. b0 + batch - 1 of the batches the operand
// maps cover (eA, eB, out and the partial buffers are then the sub-batch's own:
// the caller offsets them).  ckb > 0: K blocks per chunk instead of
// tc_chunk_blocks' choice for this shape (a sub-batch then sums in the whole
// product's order; at most 32).
cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, int M, int Nr, int Kr, int batch,
                    const int* eA, long seA, const int* eB, long seB, void* out, bool out_f64, long ldo,
                    long sbo, int* ps0, float* pbc, int* err, cudaStream_t s,
                    cudaEvent_t gemm_done = nullptr, int products = 8, int a_conv = 0, int herm = 0,
                    const float* dot_with = nullptr, double* dot_partial = nullptr, int dot_max = 0,
                    int* dot_blocks = nullptr, int b0 = 0, int ckb = 0);

// Map of an FP32 matrix [batch][rows][ld floats] (cols valid) in 32-float K
// boxes of 128 rows with 128B swizzle (ld * 4 bytes a multiple of 16).
cudaError_t make_f32_map(void* map_out, const void* base, int batch, int rows, int cols, int ld);

// Map of the FP32 matrix [batch][kdim][ld floats] whose first 2 rows floats
// of each K row are valid, read as the transpose: boxes of 16 K rows by 128
// complex rows (256 floats), no swizzle (ld * 4 bytes a multiple of 16).
cudaError_t make_f32_map_t(void* map_out, const void* base, int batch, int kdim, int rows, int ld);

// Map of a 2-D FP32 array [outer][inner] (rows stride_bytes apart, a multiple
// of 16) read as boxes of box0 (inner, box0 * 4 bytes a multiple of 16) by
// box1 rows, no swizzle, zero past the ends.
cudaError_t make_f32_map_2d(void* map_out, const void* base, long inner, long outer, long stride_bytes, int box0,
                            int box1);

// Map of a 3-D FP32 array [d2][d1][d0] (strides s1_bytes, s2_bytes, multiples
// of 16) read as boxes b0 x b1 x b2 (b0 * 4 bytes a multiple of 16), no
// swizzle, zero past the ends.
cudaError_t make_f32_map_3d(void* map_out, const void* base, long d0, long d1, long d2, long s1_bytes,
                            long s2_bytes, int b0, int b1, int b2);

// 32-wide real-K blocks per chunk of a product of this shape: the fewest
// chunks of at most 32 blocks (the exact leading sums), of equal length; a
// product split anyway takes one chunk more when it would otherwise have
// fewer than six 128 x 128 x chunk units per SM of a 152-SM part.
int tc_chunk_blocks(int M, int Nr, int Kr, int batch);

// Elements of each split-K partial buffer tc_gemm needs for this shape (0 if none).
long tc_partial_elems(int M, int Nr, int Kr, int batch);

// Row exponents of src[b][r][0..cols) (contiguous rows): e[b * rows + r], the
// smallest e with max_c max(|re|, |im|) < 2^e (0 for a zero row).
cudaError_t row_exponents_z(const double2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s);
cudaError_t row_exponents_c(const float2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s);
// Column exponents: e[b * cols + c] over r of src[b][r][c].
cudaError_t col_exponents_z(const double2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s);
cudaError_t col_exponents_c(const float2* src, long sbs, int lds, int batch, int rows, int cols, int* e,
                            cudaStream_t s);

// The three fp16 slices of the contiguous rows src[row][0..np) (rows = batch
// x rows per batch) with each row's exact exponent, found by the same kernel;
// writes the exponents to e[row].  bplanes (optional, same ldp): also the
// embedded B operand of src^H that embed_b writes for (src, conj_src,
// conj_a = 0) with these exponents (rows 2 row, 2 row + 1).
cudaError_t slice_rows_exact(const float2* src, int np, long rows, int* e, uint16_t* planes, long plane, int ldp,
                             cudaStream_t s, uint16_t* bplanes = nullptr, long bplane = 0);
// Exponents alone of the contiguous rows src[row][0..np): one warp per row,
// 16-byte loads when np is even.
cudaError_t row_exponents_rows(const float2* src, int np, long rows, int* e, cudaStream_t s);

// Embedded B operand planes (three fp16 slices) of a complex B(k, j) (K x J per batch):
//   planes[p][b][2j + c][2k + d] = slice_p(E_cd(B(k, j)))  with row exponent e[b][j]
// E = [[Br, -Bi], [Bi, Br]] (conj_a = 0) or [[Br, Bi], [Bi, -Br]] (conj_a = 1).
// B(k, j) = src[b * sbs + k * ldk + j * ldj], conjugated if conj_src; the
// source is complex128 (src_f64) or complex64.
cudaError_t embed_b(const void* src, bool src_f64, long sbs, long ldk, long ldj, bool conj_src, bool conj_a,
                    int batch, int K, int J, const int* e, uint16_t* planes, long plane, int ldp,
                    cudaStream_t s);

