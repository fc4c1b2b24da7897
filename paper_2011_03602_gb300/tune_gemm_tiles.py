"""Run the tile-width autotuner of the grouped FP64-equivalent product on
GPU 0 and write its choices as the library's built-in table
(csrc/eq_tile_table.inc); rebuild the library afterwards.

  python -m paper_2011_03602_gb300.tune_gemm_tiles [--print-only]
  python -m paper_2011_03602_gb300.tune_gemm_tiles --from-json FILE

Prints one JSON line: the chosen width per (n, k) bucket and the mean launch
time of every width (milliseconds, synthetic groups of 96 products drawn in
the bucket).  --from-json writes the table from such a line saved earlier
(no GPU needed)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "csrc", "eq_tile_table.inc")
N_LABELS = ["n<=32", "n<=64", "n<=128", "n<=256", "n<=512", "n>512"]
K_LABELS = ["k<=64", "k<=128", "k<=256", "k<=512", "k>512"]


def write_table(widths):
    lines = ["// tile widths [n bucket][k bucket]: n <= 32, 64, 128, 256, 512, larger;",
             "// k <= 64, 128, 256, 512, larger -- written by tune_gemm_tiles.py from",
             "// oo_tune_gemm_tiles on GB300 (fastest mean launch time per bucket)"]
    for row in widths:
        lines.append("{" + ", ".join(str(int(w)) for w in row) + "},")
    with open(TABLE, "w") as f:
        f.write("\n".join(lines) + "\n")


def main(argv):
    if "--from-json" in argv:
        line = open(argv[argv.index("--from-json") + 1]).read().strip().splitlines()[-1]
        d = json.loads(line)["widths"]
        write_table([[d[n][k] for k in K_LABELS] for n in N_LABELS])
        return 0
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2011_03602_gb300 import build, oo
    build.build()
    ctx = oo.oo_create(0)
    try:
        widths, ms = oo.oo_tune_gemm_tiles(ctx)
    finally:
        oo.oo_destroy(ctx)
    out = {"widths": {n: dict(zip(K_LABELS, map(int, row))) for n, row in zip(N_LABELS, widths)},
           "ms_w32_w64_w128": {n: {k: [round(float(t), 4) for t in ms[i, j]] for j, k in enumerate(K_LABELS)}
                               for i, n in enumerate(N_LABELS)}}
    print(json.dumps(out))
    if "--print-only" not in argv:
        write_table(widths)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
