// tables.cu - the tricode -> isoclass table used by IsoTricode (Fig. 5, step 2.1.4.1).
//
// A triad state is a 6-bit code over the ordered roles (u, v, w) (Sec. 3: 64 states, 16
// classes).  Bits: 1 = v->u, 2 = u->v, 4 = v->w, 8 = w->v, 16 = u->w, 32 = w->u.  Two
// 3-vertex digraphs are isomorphic exactly when their multisets of per-vertex
// (out-degree, in-degree) pairs agree, so each code is classified by its sorted
// degree-pair signature, matched against the signature of each class written from the
// class definition.
#include <algorithm>
#include <mutex>

#include "graph.cuh"

namespace tc {
namespace {

struct Sig { uint8_t p[3][2]; };   // sorted (out, in) pairs

// One signature per class, census order.  Per class: the arcs it is defined by, then the
// resulting (out, in) of each vertex.
const Sig kClassSig[16] = {
    {{{0, 0}, {0, 0}, {0, 0}}},   // 003  no arcs
    {{{0, 0}, {0, 1}, {1, 0}}},   // 012  x->y
    {{{0, 0}, {1, 1}, {1, 1}}},   // 102  x<->y
    {{{0, 1}, {0, 1}, {2, 0}}},   // 021D x->y, x->z
    {{{0, 2}, {1, 0}, {1, 0}}},   // 021U y->x, z->x
    {{{0, 1}, {1, 0}, {1, 1}}},   // 021C x->y->z
    {{{1, 0}, {1, 1}, {1, 2}}},   // 111D x<->y, z->y
    {{{0, 1}, {1, 1}, {2, 1}}},   // 111U x<->y, y->z
    {{{0, 2}, {1, 1}, {2, 0}}},   // 030T x->y, y->z, x->z
    {{{1, 1}, {1, 1}, {1, 1}}},   // 030C x->y->z->x
    {{{1, 1}, {1, 1}, {2, 2}}},   // 201  x<->y, x<->z
    {{{1, 2}, {1, 2}, {2, 0}}},   // 120D y<->z, x->y, x->z
    {{{0, 2}, {2, 1}, {2, 1}}},   // 120U y<->z, y->x, z->x
    {{{1, 1}, {1, 2}, {2, 1}}},   // 120C y<->z, x->y, z->x
    {{{1, 2}, {2, 1}, {2, 2}}},   // 210  x<->y, y<->z, x->z
    {{{2, 2}, {2, 2}, {2, 2}}},   // 300  all six arcs
};

uint8_t g_table[64];
std::once_flag g_once;
bool g_ok = false;

void derive() {
    // role indices: u = 0, v = 1, w = 2; bit b of the code is the arc kArc[b]
    const int kArc[6][2] = {{1, 0}, {0, 1}, {1, 2}, {2, 1}, {0, 2}, {2, 0}};
    bool ok = true;
    for (int code = 0; code < 64; ++code) {
        int deg[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        for (int b = 0; b < 6; ++b)
            if (code >> b & 1) { deg[kArc[b][0]][0]++; deg[kArc[b][1]][1]++; }
        int key[3];
        for (int x = 0; x < 3; ++x) key[x] = deg[x][0] * 4 + deg[x][1];
        std::sort(key, key + 3);
        int found = -1;
        for (int c = 0; c < 16; ++c) {
            bool eq = true;
            for (int x = 0; x < 3; ++x) eq &= (key[x] == kClassSig[c].p[x][0] * 4 + kClassSig[c].p[x][1]);
            if (eq) { ok &= (found < 0); found = c; }
        }
        ok &= (found >= 0);
        g_table[code] = (uint8_t)(found < 0 ? 0 : found);
    }
    g_ok = ok;
}

}  // namespace

const uint8_t* host_tricode_table() {
    std::call_once(g_once, derive);
    return g_ok ? g_table : nullptr;
}

}  // namespace tc
