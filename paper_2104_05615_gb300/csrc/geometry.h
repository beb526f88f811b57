// Host-side lattice geometry: block-major site order, neighbour tables of the
// global even/odd hop and of the local (per-block) operator, gathered links.
#pragma once

#include <cstdint>
#include <vector>

#include "dwf_internal.h"

namespace dwf {

// Tables of one lattice.  Packed (device) order of each parity: block after
// block, block-local lexicographic order inside a block, padded to Nb_pad.
//
// Local operator regions of a block (Sec. 2.3 / 3.1.2, restated with an
// L1-distance halo instead of a cubic pad): d(r) = sum over partitioned
// dimensions of the distance of r to the block.
//   interior: even sites, d = 0        (vector space of the inner solve)
//   O1      : odd sites,  d <= 1       (outputs of stages 1 and 3)
//   E2      : even sites, d <= 2       (outputs of stage 2; interior first)
// Stage tables (input indices absolute over all blocks):
//   t1: O1 -> interior (-1 outside)    t2: E2 -> O1 (-1 outside)
//   t3: O1 -> E2                       t4: interior -> O1
struct LatticeGeom {
    int L[4] = {0, 0, 0, 0}, sub[4] = {0, 0, 0, 0}, nbk[4] = {0, 0, 0, 0};
    long V = 0, Vh = 0;
    int nblk = 0;
    int Nb = 0, Nb_pad = 0;
    int O1 = 0, E2 = 0, O1_pad = 0, E2_pad = 0;
    bool antiperiodic_t = false;

    std::vector<long> even_cb;   // packed even index -> canonical cb index (lex/2), -1 padding
    std::vector<long> odd_cb;
    // global hop: even outputs <- odd inputs, odd outputs <- even inputs
    std::vector<int> nbr_e, nbr_o;          // [n*8]
    std::vector<long> lnk_e, lnk_o;         // [n*8]: link source (see link_matrix), -1 none
    // local operator
    std::vector<int> t1, t2, t3, t4;        // [nblk*region_pad*8]
    std::vector<long> lnk_O1, lnk_E2;       // [nblk*region_pad*8]

    long ne() const { return (long)nblk * Nb_pad; }
};

// A link source encodes (lex*4+mu)*2 + dagger: the matrix U_{lex,mu} or its
// adjoint.
bool build_geometry(LatticeGeom &g, const int dims[4], const int sub[4], int antiperiodic_t,
                    std::string &err);

// Compressed link rows (first two rows, 12 reals) of every entry of src,
// converted to the element type of precision p (P64 double, P32 float, else
// half).  gauge: canonical host gauge (V*4*9 complex).
void gather_links(const std::vector<long> &src, const double *gauge, Prec p,
                  std::vector<unsigned char> &out);

}  // namespace dwf
