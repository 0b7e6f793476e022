// Packing of one particle set for snapshots: the live particles of every
// slot's segment and 8 direction buckets, copied to or from six contiguous
// arrays (x, y, ux, uy, uz, w), each `total` long.  off[9 s] is slot s's
// segment offset in them and off[9 s + 1 + d] its bucket d's; counts are
// taken as min(count, capacity).  No physics: storage plumbing only.
#pragma once

#include "common.cuh"

namespace pic {

template <typename R>
cudaError_t launch_pack(const Geom &g, SoA<R> seg, const int *cnt, int cap, SoA<R> bkt,
                        const int *bcnt, Buckets bk, const long long *off, R *dst,
                        long long total, cudaStream_t s);
template <typename R>
cudaError_t launch_unpack(const Geom &g, const R *src, long long total, const long long *off,
                          SoA<R> seg, const int *cnt, int cap, SoA<R> bkt, const int *bcnt,
                          Buckets bk, cudaStream_t s);

}  // namespace pic
