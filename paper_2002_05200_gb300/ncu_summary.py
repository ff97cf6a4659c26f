"""Summarises an ncu CSV launch list (--metrics gpu__time_duration.sum --csv)
into per-kernel launches, total device time and share."""
import collections
import csv
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
         "s": 1e3, "second": 1e3}


def _short(full: str) -> str:
    """Kernel name without return type, namespaces and parameter list."""
    name = full[5:] if full.startswith("void ") else full
    for ns in ("logan::<unnamed>::", "logan::(anonymous namespace)::", "unnamed>::", "logan::"):
        if name.startswith(ns):
            name = name[len(ns):]
    depth, cut = 0, len(name)
    for i, ch in enumerate(name):
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0:
            cut = i
            break
    return name[:cut].replace("(int)", "")


def summarize(path):
    rows = list(csv.reader(open(path)))
    hi = [i for i, r in enumerate(rows) if r and r[0] == "ID"][0]
    h = rows[hi]
    ki, mi, vi, ui = (h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"),
                      h.index("Metric Unit"))
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = _short(r[ki])
        tot[name] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
        cnt[name] += 1
    T = sum(tot.values())
    out = [f"{'kernel':42s} {'launches':>8s} {'total ms':>11s} {'share':>7s}"]
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        out.append(f"{k:42s} {cnt[k]:8d} {v:11.3f} {100 * v / T:6.2f}%")
    out.append(f"{'all':42s} {sum(cnt.values()):8d} {T:11.3f}")
    return "\n".join(out)


if __name__ == "__main__":
    print(summarize(sys.argv[1]))
