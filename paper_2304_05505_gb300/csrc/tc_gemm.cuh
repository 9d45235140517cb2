// Tensor-core (tcgen05) GEMM of the mixed build: operand planes and launcher.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Three bf16 planes of one GEMM operand, each a TMA tensor map over
// [batch][rows][ld] (64-element K boxes, 128 rows, 128B swizzle).
struct TcOperand {
  alignas(64) unsigned char map[3][128];
};

// Encode the map of one bf16 plane: `rows` x `cols` valid elements per batch,
// leading dimension `ld` elements (ld * 2 bytes must be a multiple of 16).
cudaError_t make_plane_map(void* map_out, const void* base, int batch, int rows, int cols, int ld);

// out[b][m][n] (n < Nr real columns, interleaved complex) = A'[b] B'[b]^T with
// A' = A planes (M rows, Kr real K) and B' = B planes (Nr rows, Kr real K).
// FP32 output, or FP64 output when out_f64.  `err` receives a nonzero code if a
// device wait gave up.
cudaError_t tc_gemm(const TcOperand& A, const TcOperand& B, int M, int Nr, int Kr, int batch, void* out,
                    bool out_f64, long ldo, long sbo, int* err, cudaStream_t s);

// Split a complex matrix into three bf16 planes: planes[p][b][r][2c + d] of
// src[b][r][c] (rows x cols, leading dimension lds complex); ldp = plane ld.
cudaError_t split_rows_z(const double2* src, long sbs, int lds, int batch, int rows, int cols,
                         uint16_t* p0, uint16_t* p1, uint16_t* p2,
                         int ldp, cudaStream_t s);
cudaError_t split_rows_c(const float2* src, long sbs, int lds, int batch, int rows, int cols,
                         uint16_t* p0, uint16_t* p1, uint16_t* p2,
                         int ldp, cudaStream_t s);
// Transposed split: planes[p][b][c][2r + d] of src[b][r][c].
cudaError_t split_cols_z(const double2* src, long sbs, int lds, int batch, int rows, int cols,
                         uint16_t* p0, uint16_t* p1, uint16_t* p2,
                         int ldp, cudaStream_t s);

// Embedded B operand planes of a complex B(k, j) (K x J per batch):
//   planes[p][b][2j + c][2k + d] = split_p(E_cd(B(k, j)))
// with E = [[Br, -Bi], [Bi, Br]] (conj_a = 0) or [[Br, Bi], [Bi, -Br]]
// (conj_a = 1).  B(k, j) = src[b * sbs + k * ldk + j * ldj], conjugated if
// conj_src.  The source is complex128 (src_f64) or complex64.
cudaError_t embed_b(const void* src, bool src_f64, long sbs, long ldk, long ldj, bool conj_src,
                    bool conj_a, int batch, int K, int J, uint16_t* p0,
                    uint16_t* p1, uint16_t* p2, int ldp, cudaStream_t s);
