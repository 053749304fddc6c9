// Radial statistics of L1 haloes (radial.cu).
#pragma once
#include "cso_internal.cuh"

// For each L1 halo h < H, whose members are elements seg[h] .. seg[h + 1] - 1
// of epos (grouped by halo; ehal[j] is the halo of element j), fill out[h]
// from rows[h] (the centre comes from its L2max or L1 com).  Positions are in
// stored coordinates (x relative to x0).  `pinned` is 8 bytes of host memory
// for the one readback (the largest distance, which sizes the sort key).
// The shrinking-sphere fields start from each halo's nucleus, element
// hnuc[h] of nuc_pos (the group-level member positions).
int radial_run(const uint32_t* seg, const uint32_t* ehal, const int4* epos, long long na, const cso_halo* rows,
               int H, int x0, double u, const uint32_t* hnuc, const int4* nuc_pos, cso_radial* out, void* pinned,
               Workspace& ws, cudaStream_t st);
