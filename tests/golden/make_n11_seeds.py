"""Write n11_seeds.txt: the n = 11 seeds of Section 4.4, computed by the oracle alone.

Route (Section 4.4, "Enumeration for n = 11", taken over every labelled link):
  1. n = 10, m = 14: for each IDCM orbit representative (Proposition 4.3), every WPM with
     the base facet and the upper-bound-theorem cap (Algorithm 4.4, line 5);
  2. the links L: those WPMs that use all 14 vertices (Pic(L) = 4, line 9), each with the
     map of the orbit it came from. The seedness discard of line 10 is skipped, as the
     section asks (the link of a vertex of a seed need not be a seed);
  3. for each L: K on 15 vertices, vertex 14 the apex with the one nonzero vector the map
     misses, searched with conditions (1) and (2) (cone facets forced in, the other
     candidate facets through the apex forced out) and the cap;
  4. the found K that pass lines 9-12 (Pic(K) = 4, seedness), their isomorphism classes
     (canonical forms) and the PL-sphere test of Lemma 3.3 on one member per class.
Every labelled link is used, not one per isomorphism class, so every map that a link
supports is covered. The paper's Theorem for n = 11 states that exactly 4 classes remain.

Every conditioned search is also run the paper's way (the kernel sweep with its leading
coordinates fixed by conditions (1), (2) through a column echelon form); the totals of both
routes are written.

Also written: a seeded sample of 16 links with the oracle's results of their conditioned
searches (count, nodes, probes, and how many pass lines 9-12), the inputs of GPU parity
tests. Calls only the oracle (and the seeded input generators). About six minutes on 8
cores:

    python tests/golden/make_n11_seeds.py
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2301_00806_gb300 import instances as I  # noqa: E402

N_LINK, M_LINK = 10, 14
N, M = 11, 15
SAMPLE = 16
SAMPLE_SEED = 1100806


def _links_of_orbit(oi):
    rep = I.idcm_orbit_reps(N_LINK)[oi]
    f = O.candidate_facets("dual", N_LINK, M_LINK, rep)
    c, _, _, masks = O.enumerate_dfs(N_LINK, M_LINK, f, cap=O.CAP_UBT, base_facet=True,
                                     list_mode=True, capacity=1 << 17)
    rows = [masks[i] for i in range(c) if O.pic_full(M_LINK, O.masks_to_facets(f, masks[i]))]
    return c, np.asarray(rows, dtype=np.uint64)


def _conditioned(oi, rows):
    """Results of the conditioned n = 11 searches of the links `rows` (masks over the n = 10
    candidates of orbit oi): per link (count, nodes, probes, [kept complexes], and the count,
    free coordinates and kept count of the sweep with Section 4.4's initialization)."""
    rep = I.idcm_orbit_reps(N_LINK)[oi]
    f10 = O.candidate_facets("dual", N_LINK, M_LINK, rep)
    out = []
    for row in rows:
        L = O.masks_to_facets(f10, row)
        _, f, fin, fout = O.link_conditions(N, M, rep, L)
        c, nodes, probes, masks = O.enumerate_dfs(N, M, f, cap=O.CAP_UBT, forced_in=fin,
                                                  forced_out=fout, list_mode=True, capacity=256)
        kept = []
        if c:
            keep = O.filter_pic_seed(N, M, f, masks)
            kept = [tuple(O.masks_to_facets(f, masks[i])) for i in range(c) if keep[i]]
        cs, _, n_free, smasks = O.enumerate_sweep_fixed(N, M, f, cap=O.CAP_UBT, forced_in=fin,
                                                        forced_out=fout, capacity=256)
        skept = int(O.filter_pic_seed(N, M, f, smasks).sum()) if cs else 0
        out.append((c, nodes, probes, kept, cs, n_free, skept))
    return out


def _conditioned_job(args):
    return args[0], args[1], _conditioned(args[0], args[2])


def _form(K):
    return O.canonical_form(M, list(K))


def main():
    O.oracle.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(cores, 3)) as pool:
        per_orbit = pool.map(_links_of_orbit, range(len(I.idcm_orbit_reps(N_LINK))))
    line7 = sum(c for c, _ in per_orbit)
    links = [(oi, rows) for oi, (_, rows) in enumerate(per_orbit)]
    n_links = sum(len(r) for _, r in links)
    print("n = 10 line 7:", line7, "links with Pic = 4:", n_links, flush=True)

    jobs = [(oi, s, rows[s:s + 1024]) for oi, rows in links for s in range(0, len(rows), 1024)]
    with ctx.Pool(cores) as pool:
        done = pool.map(_conditioned_job, jobs, chunksize=1)
    total_wpms = sum(r[0] for _, _, rr in done for r in rr)
    kept = [K for _, _, rr in done for r in rr for K in r[3]]
    print("conditioned WPMs:", total_wpms, "after lines 9-12:", len(kept), flush=True)
    sweep_wpms = sum(r[4] for _, _, rr in done for r in rr)
    sweep_kept = sum(r[6] for _, _, rr in done for r in rr)
    free_dims = sorted({r[5] for _, _, rr in done for r in rr})
    print("by Section 4.4's initialization:", sweep_wpms, sweep_kept, free_dims, flush=True)

    with ctx.Pool(cores) as pool:
        forms = pool.map(_form, kept, chunksize=64)
    size = {}
    for fm in forms:
        size[fm] = size.get(fm, 0) + 1
    classes = sorted(size, key=lambda fm: (len(fm), fm))
    sphere = {fm: O.pl_sphere(N, M, list(fm)) for fm in classes}
    n_spheres = sum(sphere.values())
    print("classes:", len(classes), "PL spheres:", n_spheres, flush=True)

    rng = I.SplitMix64(SAMPLE_SEED)
    flat = [(oi, k) for oi, rows in links for k in range(len(rows))]
    picks = sorted(rng.below(len(flat)) for _ in range(SAMPLE))
    sample = []
    for idx in picks:
        oi, k = flat[idx]
        row = links[oi][1][k]
        c, nodes, probes, kk = _conditioned(oi, [row])[0][:4]
        sample.append((oi, row, c, nodes, probes, len(kk)))

    lines = [
        "# Section 4.4 (Enumeration for n = 11) through every labelled link; written by",
        "# make_n11_seeds.py from the oracle alone. Lines: totals; one 'class' line per",
        "# isomorphism class of the K that pass Algorithm 4.4 lines 9-12 (members, PL sphere",
        "# 0/1, facets of the oracle's canonical form as hex vertex masks); 'sample' lines: orbit",
        "# index of the n = 10 map, the link as a mask over that map's candidate facets (words",
        "# 0.. in hex), and the oracle's count, nodes, probes and kept (lines 9-12) of its",
        "# conditioned n = 11 search.",
        f"line7_n10 {line7}",
        f"links {n_links}",
        f"conditioned_wpms {total_wpms}",
        f"pic_seed {len(kept)}",
        f"sweep_fixed_wpms {sweep_wpms}",
        f"sweep_fixed_pic_seed {sweep_kept}",
        f"sweep_fixed_free_max {max(free_dims)}",
        f"classes {len(classes)}",
        f"spheres {n_spheres}",
    ]
    for fm in classes:
        lines.append(" ".join(["class", str(size[fm]), str(int(sphere[fm]))] +
                              [f"{x:04x}" for x in fm]))
    for oi, row, c, nodes, probes, nk in sample:
        lines.append(" ".join(["sample", str(oi)] + [f"{int(x):016x}" for x in row] +
                              [str(c), str(nodes), str(probes), str(nk)]))
    with open(os.path.join(HERE, "n11_seeds.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
