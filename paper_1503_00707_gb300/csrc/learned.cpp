// Host geometry of the local Knudsen sensor: weighted least-squares gradient
// coefficients per cell from the interior faces of the mesh.
#include "learned.hpp"

#include <cmath>
#include <utility>

namespace dvm {

namespace {

// Solve the n x n system M x = r (n <= 3) by Gaussian elimination with
// partial pivoting; false on a zero pivot.
bool small_solve(int n, double M[9], double r[3], double x[3])
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int q = c + 1; q < n; q++)
            if (std::fabs(M[q * n + c]) > std::fabs(M[piv * n + c])) piv = q;
        if (!(std::fabs(M[piv * n + c]) > 0.0)) return false;
        if (piv != c) {
            for (int k = 0; k < n; k++) std::swap(M[c * n + k], M[piv * n + k]);
            std::swap(r[c], r[piv]);
        }
        for (int q = c + 1; q < n; q++) {
            const double f = M[q * n + c] / M[c * n + c];
            for (int k = c; k < n; k++) M[q * n + k] -= f * M[c * n + k];
            r[q] -= f * r[c];
        }
    }
    for (int q = n - 1; q >= 0; q--) {
        double s = r[q];
        for (int k = q + 1; k < n; k++) s -= M[q * n + k] * x[k];
        x[q] = s / M[q * n + q];
    }
    return true;
}

}  // namespace

void build_kn_stencil(const Mesh &m, KnStencil &out)
{
    const int dim = m.spec.dim;
    const int64_t nc = (int64_t)m.leaf_of_cell.size();
    std::vector<double> xc(3 * (size_t)nc);
    for (int64_t c = 0; c < nc; c++) {
        const Leaf &l = m.leaves[(size_t)m.leaf_of_cell[c]];
        const double h = std::ldexp(1.0, -l.lev);
        for (int d = 0; d < 3; d++) xc[3 * c + d] = d < dim ? (l.i[d] + 0.5) * h : 0.5;
    }
    // neighbour lists (both directions of every interior face between cells)
    out.start.assign((size_t)nc + 1, 0);
    const size_t nf = m.fm.size();
    for (size_t q = 0; q < nf; q++) {
        const int64_t a = m.cell_of_leaf[(size_t)m.fm[q]], b = m.cell_of_leaf[(size_t)m.fp[q]];
        if (a < 0 || b < 0) continue;
        out.start[(size_t)a + 1]++;
        out.start[(size_t)b + 1]++;
    }
    for (int64_t c = 0; c < nc; c++) out.start[(size_t)c + 1] += out.start[(size_t)c];
    const size_t ne = (size_t)out.start[(size_t)nc];
    out.nb.assign(ne, 0);
    std::vector<double> area(ne, 0.0);
    std::vector<int32_t> fill(out.start.begin(), out.start.end() - 1);
    for (size_t q = 0; q < nf; q++) {
        const int64_t a = m.cell_of_leaf[(size_t)m.fm[q]], b = m.cell_of_leaf[(size_t)m.fp[q]];
        if (a < 0 || b < 0) continue;
        out.nb[(size_t)fill[(size_t)a]] = (int32_t)b;
        area[(size_t)fill[(size_t)a]++] = m.farea[q];
        out.nb[(size_t)fill[(size_t)b]] = (int32_t)a;
        area[(size_t)fill[(size_t)b]++] = m.farea[q];
    }
    out.coef.assign(3 * ne, 0.0);
    std::vector<double> dv(3 * ne, 0.0), wv(ne, 0.0);
    for (int64_t c = 0; c < nc; c++) {
        double N[9] = {0};
        for (int32_t e = out.start[(size_t)c]; e < out.start[(size_t)c + 1]; e++) {
            const int64_t nb = out.nb[(size_t)e];
            double d[3] = {0, 0, 0}, d2 = 0.0;
            for (int k = 0; k < dim; k++) {
                d[k] = xc[3 * nb + k] - xc[3 * c + k];
                if (m.spec.bc[2 * k] == DVM_BC_PERIODIC) {
                    if (d[k] > 0.5) d[k] -= 1.0;
                    if (d[k] < -0.5) d[k] += 1.0;
                }
                d2 += d[k] * d[k];
            }
            const double w = area[(size_t)e] / d2;
            wv[(size_t)e] = w;
            for (int k = 0; k < 3; k++) dv[3 * (size_t)e + k] = d[k];
            for (int r = 0; r < dim; r++)
                for (int k = 0; k < dim; k++) N[r * dim + k] += w * d[r] * d[k];
        }
        // coefficient of neighbour e: w_e N^{-1} d_e (zero if N is singular)
        for (int32_t e = out.start[(size_t)c]; e < out.start[(size_t)c + 1]; e++) {
            double M[9], r[3], x[3] = {0, 0, 0};
            for (int k = 0; k < dim * dim; k++) M[k] = N[k];
            for (int k = 0; k < dim; k++) r[k] = wv[(size_t)e] * dv[3 * (size_t)e + k];
            if (!small_solve(dim, M, r, x)) break;
            for (int k = 0; k < dim; k++) out.coef[3 * (size_t)e + k] = x[k];
        }
    }
}

}  // namespace dvm
