// me_batch_types.h -- the stream and work tables of the multi-stream
// persistent forms, shared by the batch/server kernels and the pipelined full
// search.  Internal.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "me_search.cuh"

namespace me {

struct BStream {  // per-run arguments of one stream (copied to the device each run)
  const uint8_t* cur;
  const uint8_t* ref;
  const int16_t* prev;
  int16_t* mv;
  uint32_t* J;
  uint8_t* mask;
  uint32_t* sad;
  uint32_t* load;
  uint32_t lam;
  int32_t alpha, beta, gnum, gden, qp, refine;
};

struct BShape {  // fixed per stream
  int W, H, p;
  PadGeom pg;
  uint8_t* refpad;
  uint32_t* intra;
  unsigned long long* flags;  // per block: epoch + final vector (pub_word)
  long long pad_base;  // first 16-byte chunk of this stream in the flat pad index
  int blk_base;        // first block of this stream in the flat block index
  // speculative full searches of the ACBM step (null: none): per block the
  // search's key and the state word (searched / PBM failed), cleared each step
  unsigned long long* bkey;
  int* bstate;
};

struct BFsEntry {  // FSBM: one group of adjacent blocks, G threads per block
  int stream, by, bx0, nb, G;
};

// The pipelined full search at any p <= 64 (k_fsbm_pipe_tab): groups of
// pipe_tab_bpc(N, p) adjacent blocks of one block row.  The batch form takes
// the batch's stream and group tables (nb <= pipe_tab_bpc of the stream's
// p), claims groups from *ctr (zero before the launch) and reports a wait
// that gave up in *err.
bool pipe_tab_applies(int N, int M, int p);
int pipe_tab_bpc(int N, int p);
int pipe_tab_T(int N, int M);
int launch_pipe_tab_seq(const uint8_t* const* frames, int K, int W, int H, int N, int M, int p,
                        uint32_t lam, int16_t* mv_out, uint32_t* J_out, uint32_t* sad_out,
                        cudaStream_t s);
int launch_pipe_tab_batch(int N, int M, const BShape* shp, const BStream* st, const BFsEntry* ent,
                          int nent, int* ctr, int* err, cudaStream_t s);

}  // namespace me
