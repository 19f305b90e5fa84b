// The molecule of batch j in a chunk: for a grouped chunk (several molecules in one combined
// plan) the entry of the molecule table, otherwise the chunk's own P, V_acc, nbf and functional
// (and no double-float P planes: the tensor-core kernels then take the chunk's).
#pragma once

#include "internal.h"

namespace gbxc {

__device__ __forceinline__ MolRef mol_of(const ChunkArgs &a, int j) {
    if (a.batch_mol) return a.mols[a.batch_mol[j]];
    MolRef r;
    r.P = a.P;
    r.Vacc = a.Vacc;
    r.pdf = nullptr;
    r.nbf = a.nbf;
    r.functional = a.functional;
    return r;
}

}  // namespace gbxc
