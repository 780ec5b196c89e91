"""Independent brute-force restatement of one simulation step, for tiny cases.

It follows the same rules as the oracle (Algorithm 1 with the readings listed
in the oracle's header) but shares none of its structure: there is no lane
map, no double buffer, no erase pass and no claim array.  Vehicles are plain
records; a leader, a free cell or a gap is found by searching the other
vehicles' positions; entry conflicts are settled by sorting the requests.
All arithmetic is numpy float32 scalars (IEEE binary32, one rounding per
operation, no fused multiply-add), in the order the rules state it.
"""
from __future__ import annotations

import math

import numpy as np

F = np.float32
WAITING, ACTIVE, ARRIVED = 0, 1, 2
M64 = (1 << 64) - 1


def splitmix64_mix(z: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014)."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def unit24(h: int) -> np.float32:
    return F(F(h >> 40) * F(1.0 / 16777216.0))


def speed_byte(v: np.float32) -> int:
    return int(min(float(v), 254.0))


def fmax0(t):
    return t if t > F(0) else F(0)


class BruteForce:
    def __init__(self, net: dict, params: dict, vehicle_types: list | None = None):
        p = {k: F(v) if isinstance(v, float) else v for k, v in params.items()}
        self.p = p
        # vehicle types: each its own IDM parameters and top speed; without
        # them one type with the run parameters and no top speed of its own
        tys = vehicle_types or [dict(a=p["a"], b=p["b"], s0=p["s0"], T=p["T"], vmax=254.0)]
        self.types = [dict(a=F(t["a"]), s0=F(t["s0"]), T=F(t["T"]), vmax=F(t["vmax"]),
                           tsab=F(2.0 * math.sqrt(float(F(t["a"])) * float(F(t["b"]))))) for t in tys]
        self.src = [int(a) for a in net["edge_src"]]
        self.dst = [int(a) for a in net["edge_dst"]]
        self.ncell = [max(1, int(math.ceil(float(F(a))))) for a in net["edge_len"]]
        self.v0 = [F(a) for a in net["edge_vmax"]]
        self.lanes = [int(a) for a in net["edge_lanes"]]
        self.green = [int(a) for a in net["node_green"]]
        ne = len(self.src)
        ins = {}
        for e in range(ne):
            ins.setdefault(self.dst[e], []).append(e)
        rank = net.get("edge_approach_rank")
        self.arank = [0] * ne
        for node, es in ins.items():
            for j, e in enumerate(sorted(es)):
                self.arank[e] = int(rank[e]) if rank is not None else j
        self.nphase = {node: 1 + max(self.arank[e] for e in es) for node, es in ins.items()}
        outs = {}
        for e in range(ne):
            outs.setdefault(self.src[e], []).append(e)
        self.orank = [0] * ne
        self.nout = {node: len(es) for node, es in outs.items()}
        for node, es in outs.items():
            for j, e in enumerate(sorted(es)):
                self.orank[e] = j
        self.two_sqrt_ab = F(2.0 * math.sqrt(float(p["a"]) * float(p["b"])))
        self.k = 0

    def load(self, depart_step, routes, vtypes=None):
        n = len(depart_step)
        order = sorted(range(n), key=lambda j: int(depart_step[j]))  # stable
        self.vid = [0] * n
        self.veh = []
        for i, j in enumerate(order):
            self.vid[j] = i
            self.veh.append(dict(id=i, dep=int(depart_step[j]), route=[int(e) for e in routes[j]],
                                 ty=self.types[int(vtypes[j]) if vtypes is not None else 0],
                                 status=WAITING, e=None, r=0, lane=0, x=F(0), v=F(0), t_enter=0,
                                 dep_act=0xFFFFFFFF, arr=0xFFFFFFFF))

    # ---- rules
    def is_green(self, e, k):
        node = self.dst[e]
        G = self.green[node]
        if G == 0:
            return True
        return (k // G) % self.nphase[node] == self.arank[e]

    def tl_for(self, edge, nxt):
        return (self.orank[nxt] * self.lanes[edge]) // self.nout[self.dst[edge]]

    def idm(self, ty, v, vf, s, v0):
        p = self.p
        dv = F(v - vf)
        z = F(F(v * ty["T"]) + F(F(v * dv) / ty["tsab"]))
        s_star = F(ty["s0"] + fmax0(z))
        r = F(v / v0)
        q = F(s_star / s)
        acc = F(ty["a"] * F(F(F(1.0) - F(F(r * r) * F(r * r))) - F(q * q)))
        return fmax0(F(v + F(acc * p["dt"])))

    def cell(self, w):
        return int(w["x"])

    def occupants(self):
        occ = {}
        for w in self.veh:
            if w["status"] == ACTIVE:
                key = (w["e"], w["lane"], self.cell(w))
                assert key not in occ, "two vehicles in one cell"
                occ[key] = w
        return occ

    def entry_pref(self, veh, q, occ):
        route = veh["route"]
        en = route[q]
        nl = self.lanes[en]
        tl = self.tl_for(en, route[q + 1]) if q + 1 < len(route) else 0
        cands = sorted(range(nl), key=lambda l: (abs(l - tl), l))
        for l in cands:
            if (en, l, 0) not in occ:
                return l
        return None

    def step(self):
        k = self.k
        p = self.p
        occ = self.occupants()
        active = [w for w in self.veh if w["status"] == ACTIVE]
        plan = {}
        requests = []  # (edge, lane, id)
        for w in active:
            e, ln, x, v = w["e"], w["lane"], w["x"], w["v"]
            ncell = self.ncell[e]
            L = F(ncell)
            c = self.cell(w)
            ahead = [cc for (ee, ll, cc) in occ if ee == e and ll == ln and cc > c]
            cf = min(ahead) if ahead else None
            ty = w["ty"]
            vfree = min(self.v0[e], ty["vmax"])  # the edge limit, or the type's top speed if lower
            dfront = F(F(F(2.0) * p["dt"]) * v)
            if cf is not None and F(F(cf) - x) <= dfront:
                vn = self.idm(ty, v, F(speed_byte(occ[(e, ln, cf)]["v"])), F(F(cf) - x), vfree)
            else:
                vn = vfree
            xn = F(x + F(vn * p["dt"]))
            if cf is not None:
                lim = F(F(cf) - ty["s0"])
                if xn > lim:
                    xn = x if x > lim else lim
                    vn = F(0)
            last = w["r"] == len(w["route"]) - 1
            if xn >= L:
                if last:
                    plan[w["id"]] = ("arrive", xn, vn, None)
                elif not self.is_green(e, k):
                    plan[w["id"]] = ("hold", xn, vn, None)
                else:
                    l = self.entry_pref(w, w["r"] + 1, occ)
                    if l is None:
                        plan[w["id"]] = ("hold", xn, vn, None)
                    else:
                        plan[w["id"]] = ("cross", xn, vn, l)
                        requests.append((w["route"][w["r"] + 1], l, w["id"]))
                continue
            kind, d = "stay", 0
            draw = unit24(splitmix64_mix(int(p["seed"]) ^ ((w["id"] * 0x9E3779B97F4A7C15) & M64)
                                         ^ ((k * 0xD1B54A32D192ED03) & M64)))
            must = False  # inside the mandatory lane-change zone of its next movement
            if self.lanes[e] > 1 and not last:
                tl = self.tl_for(e, w["route"][w["r"] + 1])
                if tl != ln:
                    d = 1 if tl > ln else -1
                    xrem = F(L - x)
                    must = xrem < p["x0"]
                    if (d > 0) == (k % 2 == 1):
                        m = F(0) if xrem >= p["x0"] else F(F(1.0) - F(xrem / p["x0"]))
                        if draw < m:
                            kind = "intend"
            # discretionary change: held up by a slower leader, a longer gap in
            # the lane of this step's direction (up on odd steps)
            if kind == "stay" and not must and self.lanes[e] > 1 and p.get("dlc_prob", 0.0) > 0.0:
                d = 1 if k % 2 == 1 else -1
                ln2 = ln + d
                blocked = (cf is not None and vn < vfree
                           and F(speed_byte(occ[(e, ln, cf)]["v"])) < vfree)
                if blocked and 0 <= ln2 < self.lanes[e]:
                    lead = [cc for cc in range(c, min(c + 63, ncell - 1) + 1) if (e, ln2, cc) in occ]
                    pays = not lead or F(F(lead[0]) - F(cf)) >= F(p["dlc_gain"])
                    if pays and draw < F(p["dlc_prob"]):
                        kind = "intend"
            plan[w["id"]] = (kind, xn, vn, d if kind == "intend" else 0)
        # departures: lowest waiting id per first edge, if its time has come
        heads = {}
        for w in self.veh:
            if w["status"] == WAITING:
                e0 = w["route"][0]
                if e0 not in heads or w["id"] < heads[e0]["id"]:
                    heads[e0] = w
        dep_req = {}
        for e0, w in heads.items():
            if w["dep"] <= k:
                l = self.entry_pref(w, 0, occ)
                if l is not None:
                    dep_req[w["id"]] = l
                    requests.append((e0, l, w["id"]))
        winners = {}
        for (e, l, i) in sorted(requests):
            winners.setdefault((e, l), i)  # smallest id per slot comes first
        won = set(winners.values())
        # outcome positions for k+1 (reservations)
        reserved = {}
        new_state = {}
        for w in active:
            kind, xn, vn, extra = plan[w["id"]]
            e = w["e"]
            if kind == "cross" and w["id"] in won:
                en = w["route"][w["r"] + 1]
                new_state[w["id"]] = ("move", en, w["r"] + 1, extra, F(0), vn)
                reserved[(en, extra, 0)] = w["id"]
            elif kind in ("cross", "hold"):
                lim = F(F(self.ncell[e]) - F(1.0))
                xh = w["x"] if w["x"] > lim else lim
                new_state[w["id"]] = ("held", e, w["r"], w["lane"], xh, F(0))
                reserved[(e, w["lane"], int(xh))] = w["id"]
            elif kind == "arrive":
                new_state[w["id"]] = ("arrived",)
            else:
                new_state[w["id"]] = ("stay", e, w["r"], w["lane"], xn, vn)
                reserved[(e, w["lane"], int(xn))] = w["id"]
        for i, l in dep_req.items():
            if i in won:
                reserved[(self.veh[i]["route"][0], l, 0)] = i
        # lane changes, all judged against the same occupancy and reservations
        accepted = {}
        for w in active:
            kind, xn, vn, d = plan[w["id"]]
            if kind != "intend":
                continue
            e = w["e"]
            ln2 = w["lane"] + d
            c0 = self.cell(w)
            cn = int(xn)
            same = [(cc, o) for (ee, ll, cc), o in occ.items() if ee == e and ll == ln2]
            lead = [cc for cc, o in same if c0 <= cc <= c0 + 63]
            lag = [cc for cc, o in same if c0 - 64 <= cc < c0]
            eps_a = eps_b = F(0)
            if p["eps_amp"] > F(0):
                h = splitmix64_mix(int(p["seed"]) ^ ((w["id"] * 0x9E3779B97F4A7C15) & M64)
                                   ^ ((k * 0xD1B54A32D192ED03) & M64))
                eps_a = F(p["eps_amp"] * F(F(F(2.0) * unit24(splitmix64_mix(h ^ 0x632BE59BD9B4E019))) - F(1.0)))
                eps_b = F(p["eps_amp"] * F(F(F(2.0) * unit24(splitmix64_mix(h ^ 0x8CB92BA72F3D8DD7))) - F(1.0)))
            ok = True
            if lead:
                ca = min(lead)
                va = F(speed_byte(occ[(e, ln2, ca)]["v"]))
                G_lead = F(F(p["g_a"] + fmax0(F(F(p["alpha_i"] * vn) - F(p["alpha_a"] * va)))) + eps_a)
                ok = ok and F(F(ca) - xn) >= G_lead
            if lag:
                cb = max(lag)
                vb = F(speed_byte(occ[(e, ln2, cb)]["v"]))
                G_lag = F(F(p["g_b"] + fmax0(F(F(p["alpha_b"] * vb) - F(p["alpha_i"] * vn)))) + eps_b)
                ok = ok and F(xn - F(cb)) >= G_lag
            ok = ok and cn >= 1 and (e, ln2, cn) not in reserved
            if ok:
                accepted[w["id"]] = ln2
        # apply
        for w in active:
            ns = new_state[w["id"]]
            if ns[0] == "arrived":
                w["status"] = ARRIVED
                w["arr"] = k + 1
                continue
            tag, e, r, lane, x, v = ns
            if tag == "move":
                w["t_enter"] = k + 1
            w["e"], w["r"], w["lane"], w["x"], w["v"] = e, r, accepted.get(w["id"], lane), x, v
        for i, l in dep_req.items():
            if i in won:
                w = self.veh[i]
                w.update(status=ACTIVE, e=w["route"][0], r=0, lane=l, x=F(0), v=F(0), t_enter=k + 1,
                         dep_act=k + 1)
        self.occupants()  # asserts at most one vehicle per cell
        self.k = k + 1

    def state(self):
        n = len(self.veh)
        out = {"x": np.zeros(n, np.float32), "v": np.zeros(n, np.float32), "edge": np.full(n, 0xFFFFFFFF, np.uint32),
               "lane": np.zeros(n, np.uint8), "ridx": np.zeros(n, np.uint32), "status": np.zeros(n, np.uint8)}
        for w in self.veh:
            i = w["id"]
            out["status"][i] = w["status"]
            if w["status"] == ACTIVE:
                out["x"][i], out["v"][i], out["edge"][i] = w["x"], w["v"], w["e"]
                out["lane"][i], out["ridx"][i] = w["lane"], w["r"]
        return out
