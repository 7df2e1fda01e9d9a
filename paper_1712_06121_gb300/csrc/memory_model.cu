// The memory model of Section 2.3's memory layout: bytes per image of the
// arrays a CUBE image keeps, as functions of the code widths, the image's
// coarse mesh, its buffer depth, its tiling and the inhomogeneity margins
// (Eqs. npmax, nptile, Mp_particle, Mp_coarse, Mp_fine).  Host code.
//
// Readings where the equations and the worked table (Table t.memory) differ:
//  * the tile arrays chi*_d, nu*_d carry the buffer factor (1 + 2 N_b/N_t)^3
//    as well: Eq. nptile omits it, the table's 0.872 bpp includes it;
//  * the fine force kernel K_f covers one tile of R N_e fine cells a side
//    (N_e = N_t + 2 N_b), in r2c layout (R N_e / 2 + 1 planes): Eq. Mp_fine's
//    N_t^-3 cannot give the table's 1.06 GB, this does;
//  * rho_c and v_c cover the image's M_t^3 extended tiles, (N_e M_t)^3
//    coarse cells; the coarse kernel K_c covers the image's (N_c/M_g)^3
//    cells, 3 components of 4 bytes, half of them stored (Eq. Mp_coarse).
#include <cmath>
#include <cstdint>

#include "cube.h"

namespace cube {
cube_status served_fail(cube_status s, const char* msg);
}

extern "C" cube_status cube_memory_model(const cube_memory_config* cfg, cube_memory_layout* out) {
    using cube::served_fail;
    if (!cfg || !out) return served_fail(CUBE_E_ARG, "NULL argument");
    const cube_memory_config& c = *cfg;
    if (c.x_bytes < 1 || c.x_bytes > 2 || c.v_bytes < 1 || c.v_bytes > 2)
        return served_fail(CUBE_E_ARG, "x_bytes and v_bytes must be 1 or 2");
    if (c.id_bytes != 0 && c.id_bytes != 1 && c.id_bytes != 2 && c.id_bytes != 4)
        return served_fail(CUBE_E_ARG, "id_bytes must be 0, 1, 2 or 4");
    if (c.ratio < 1 || c.coarse_per_image < 1 || c.tiles < 1 || c.buffer < 0)
        return served_fail(CUBE_E_ARG, "ratio, coarse_per_image, tiles must be >= 1 and buffer >= 0");
    if (c.coarse_per_image % c.tiles != 0) return served_fail(CUBE_E_ARG, "tiles must divide coarse_per_image");
    if (!(c.eps_image >= 0.0) || !(c.eps_tile >= 0.0) || !(c.particles_per_image > 0.0))
        return served_fail(CUBE_E_ARG, "eps_image, eps_tile must be >= 0 and particles_per_image > 0");
    const double Nt = (double)(c.coarse_per_image / c.tiles);       // coarse cells per tile side
    const double Ne = Nt + 2.0 * c.buffer;                          // extended tile side
    const double Mt = (double)c.tiles;
    const double buf = std::pow(1.0 + 2.0 * c.buffer / Nt, 3);
    const double p_max = c.particles_per_image * buf * (1.0 + c.eps_image);           // Eq. npmax
    const double p_tile = c.particles_per_image * buf * (1.0 + c.eps_tile) / (Mt * Mt * Mt);
    const double code = 3.0 * c.x_bytes + 3.0 * c.v_bytes;
    const double cells = std::pow(Ne * Mt, 3);
    const double nf = c.ratio * Ne;                                 // fine cells per extended tile side
    out->chi_nu = code * p_max;
    out->chi_nu_tile = code * p_tile;
    out->ids = c.id_bytes * (p_max + p_tile);
    out->rho_c = 4.0 * cells;
    out->v_c = 12.0 * cells;
    out->k_c = 12.0 * std::pow((double)c.coarse_per_image, 3) / 2.0;
    out->k_f = 12.0 * (std::floor(nf / 2.0) + 1.0) * nf * nf;
    out->total = out->chi_nu + out->chi_nu_tile + out->ids + out->rho_c + out->v_c + out->k_c + out->k_f;
    return CUBE_OK;
}
