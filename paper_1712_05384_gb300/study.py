"""Ordering study (Sec. IV.A-B, App. E; Figs. 4-6): treewidth bounds of grid
circuits as a function of depth, all computed by the library's planner.

For each circuit: the induced width of the vertical order on the graphical
model (Fig. 4), of the min-fill order on the graphical model (Fig. 5; the
paper used QuickBB, a third-party search, for its upper bounds), and of the
min-fill order on the line graph of the circuit's tensor network (Fig. 6).
Widths are reported as treewidth bounds, i.e. largest clique - 1, the
convention of the paper's figures.  Only host code runs (no GPU).

    python -m paper_1712_05384_gb300.study 6x6 6x7 7x7 --depths 10 15 20 25 30 35 40
"""
import argparse

from ._lib import ORDER_MINFILL, ORDER_VERTICAL, Circuit, Model, Plan


def widths(rows, cols, depth, seed=0):
    c = Circuit.grid(rows, cols, depth, seed)
    m = Model(c)
    vert = Plan(m, order_kind=ORDER_VERTICAL).info.max_clique - 1
    mf = Plan(m, order_kind=ORDER_MINFILL).info.max_clique - 1
    segments, lg = c.line_graph_width()
    return {"grid": f"{rows}x{cols}", "depth": depth, "seed": seed, "vertical": vert, "min_fill": mf,
            "line_graph": lg - 1, "segments": segments}


def study(sizes, depths, seed=0):
    return [widths(r, c, d, seed) for (r, c) in sizes for d in depths]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("sizes", nargs="*", default=["6x6", "6x7", "7x7"])
    ap.add_argument("--depths", type=int, nargs="*", default=[10, 15, 20, 25, 30, 35, 40])
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    sizes = [tuple(int(x) for x in s.split("x")) for s in a.sizes]
    print("| grid | depth | vertical (Fig. 4) | min-fill (Fig. 5) | line graph (Fig. 6) |")
    print("|---|---|---|---|---|")
    for r in study(sizes, a.depths, a.seed):
        print(f"| {r['grid']} | {r['depth']} | {r['vertical']} | {r['min_fill']} | {r['line_graph']} |")


if __name__ == "__main__":
    main()
