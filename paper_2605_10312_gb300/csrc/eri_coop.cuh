// Launch arguments of the team-cooperative executor (eri_coop.cu), shared
// with the runtime that fills them in (eri_runtime.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "eri_digest.cuh"

struct EriCoopArgs {
  const uint4* __restrict__ ph1;      // Phase-1 descriptors, waves of steps x T
  const uint32_t* __restrict__ steps1;
  const uint4* __restrict__ ph2;      // Phase-2 descriptors
  const uint32_t* __restrict__ steps2;
  const double* __restrict__ c2s;     // transform coefficient table
  double* __restrict__ gvals;         // unused: every value slot is in shared memory
  double* __restrict__ gH;            // [team][nh] when H is not in shared memory
  int32_t nw1, nw2;
  int32_t nh, nslot, L;
  int32_t smem_slots;                 // value slots held in shared memory
  int32_t h_in_smem;
  int32_t nteams;                     // teams in the grid
  int32_t batch;                      // coefficient rows per team (1..ERI_COOP_BATCH)
  int32_t single;                     // every quartet has one primitive quartet: the rows of
                                      // `batch` consecutive quartets of a team are computed together
};

// A class program of the team-cooperative tier as the persistent launch
// finds it (device pointers of its descriptor streams and its sizes).
struct EriCoopProgDesc {
  const uint4* ph1;
  const uint32_t* steps1;
  const uint4* ph2;
  const uint32_t* steps2;
  int32_t nw1, nw2, nh, nslot, L, pad;
};

// One item of a persistent launch's work list: records [first, first +
// count) of the plan's record array, all of program `prog`, evaluated by
// `teams` teams of T lanes of one block.
struct EriWorkItem {
  int32_t prog;
  int32_t first, count;
  int16_t T, teams;
  int8_t hsm, vote, single, pad;
  int32_t batch;
};

// Coulomb/exchange digestion fused into the persistent launch: after the
// last part of a quartet has reached its block, the team that finished it
// digests the block (still in L2) into J and K.
struct EriFuse {
  EriDigestArgs jk;          // blocks = the plan's output; list / nlist unused
  const int32_t* rec_q;      // user quartet of each record
  const int32_t* nparts;     // parts of each user quartet
  int32_t* done;             // parts finished per user quartet, zeroed before the launch
  int32_t on;                // 0: no digestion
  int32_t pad;
};

struct EriPersistArgs {
  const EriWorkItem* items;
  const EriCoopProgDesc* progs;
  int32_t* next;             // item counter, zeroed before the launch
  int32_t nitems;
  int32_t pad;
  double* gH;                // team-private accumulators of the items that keep H in global memory
  int64_t gh_per_block;      // elements of gH per block
  const double* c2s;
  EriFuse fuse;
};

